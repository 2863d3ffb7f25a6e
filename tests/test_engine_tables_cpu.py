"""Host-side layout of the line engine's per-stage twiddle tables
(fft_engine.cuh): for every stage span M = NS R up to 4096 and radix R in
{2, 4, 8, 16} (NS >= 2), the table of M entries starts at stage_tw_offset(M, R)
and all of them fit, without overlap, in the kStageTwiddles entries below the
power-of-two pyramid.  A host-only probe is compiled with nvcc (no GPU needed).
"""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1805_07801_gb300", "csrc")

PROBE = r"""
#include <cstdio>
#include "fft_engine.cuh"
int main() {
  std::printf("%d\n", fftk::kStageTwiddles);
  for (int M = 4; M <= 4096; M *= 2)
    for (int R = 2; R <= 16 && R <= M / 2; R *= 2) std::printf("%d %d %d\n", M, R, fftk::stage_tw_offset(M, R));
  return 0;
}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_stage_tables_fit_and_do_not_overlap(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "probe.cu"
    src.write_text(PROBE)
    exe = tmp_path / "probe"
    # built for the library's target, whose engine uses sm_100+ paired FP32
    # instructions; the probe itself runs on the host only
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC, str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    total = int(out[0])
    spans = []
    for line in out[1:]:
        if not line.strip():
            continue
        M, R, off = (int(v) for v in line.split())
        spans.append((off, off + M, M, R))
    # every (M, R) pair a stage can take is present
    assert len(spans) == sum(min(4, m - 1) for m in range(2, 13))
    spans.sort()
    assert spans[0][0] >= 0 and spans[-1][1] <= total
    for a, b in zip(spans, spans[1:]):
        assert a[1] <= b[0], (a, b)
