"""Element-by-element parity at the full sizes of the workloads, in the launch
configurations the benchmark times: the 1024^3 R2C / C2R pair (FP32 and
split-FP16 plans) against the FP64 oracle over every coefficient and every
point, the 512^3 right-hand side of the decaying-turbulence workload against
the oracle, and the 1024^3 right-hand side (the n = 1024 instantiations of the
fused kernels) against the oracle through a band-limited state.

Tolerances (FP32 unit roundoff u = 2^-24):
* FFT pair, FP32: relative L2 <= 2e-6 and 1e-5 * max|F| per element (a
  Cooley-Tukey transform with correctly rounded twiddles errs by at most
  ~u log2(N^3) = 1.8e-6 at 1024^3).
* FFT pair, split FP16: relative L2 <= 1e-5 (each tensor-core stage drops
  x_lo W_lo, 2^-22 relative).
* right-hand side: relative L2 <= 1e-5 in FP32 (nine transforms, products and
  the projection), 3e-5 with the split-FP16 passes.

The band-limited check (Sec. 2.2, the 2/3 rule): a field whose modes satisfy
|k_x|, |k_y|, |k_z| <= 85 has products with |k_i| <= 170.  On a 512^3 grid
the 2/3 rule keeps |k_i| <= 170 and the aliases of those products land at
|k_i| >= 342, outside the kept set; on a 1024^3 grid it keeps |k_i| <= 341.
So the dealiased, projected right-hand side of that field is the same set of
Fourier coefficients on both grids (the truncated convolution itself), and
the oracle's 512^3 result fixes every 1024^3 coefficient: equal on the modes
the 512^3 grid holds, zero on all the others.

Measured errors are printed ("MEASURED ...") for the record.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import empty_c64, empty_real, stream, sync

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fk():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07801_gb300 import build as b

    b.build()
    import paper_1805_07801_gb300 as m

    return m


# ----------------------------------------------------------- host helpers --
def _sums(a, b):
    """(sum |a - b|^2, sum |b|^2, max |a - b|, max |b|), slice by slice of the
    leading axis so that no full-size FP64 temporary is formed."""
    num = den = 0.0
    dmax = bmax = 0.0
    for i in range(a.shape[0]):
        ai = np.asarray(a[i], dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
        bi = np.asarray(b[i], dtype=ai.dtype)
        d = np.abs(ai - bi)
        num += float(np.sum(d * d))
        bb = np.abs(bi)
        den += float(np.sum(bb * bb))
        dmax = max(dmax, float(d.max()))
        bmax = max(bmax, float(bb.max()))
    return num, den, dmax, bmax


def _compare(a, b):
    num, den, dmax, bmax = _sums(a, b)
    return float(np.sqrt(num / den)), dmax / bmax


def _c64_to_host(t) -> np.ndarray:
    return np.ascontiguousarray(t.cpu().numpy()).view(np.complex64)[..., 0]


def _dev_real(a):
    import torch

    return torch.from_numpy(a).to("cuda:0")


def _dev_c64(a):
    import torch

    return torch.from_numpy(a.view(np.float32).reshape(a.shape + (2,))).to("cuda:0")


# ------------------------------------------------------------- FFT 1024^3 --
N_FFT = 1024


@pytest.fixture(scope="module")
def pair1024(oracle_mod):
    """The 1024^3 pair workload: normal(0, 1) values of seed 0 rounded to FP32;
    the oracle's spectrum of that FP32 field, its complex64 rounding, and the
    oracle's inverse of the rounded spectrum."""
    n = N_FFT
    f64 = synth.normal(0, 0, (n, n, n))
    f32 = f64.astype(np.float32)
    f64[...] = f32  # the oracle sees exactly the FP32 input
    Fo = oracle_mod.rfft3(f64)
    del f64
    F32 = Fo.astype(np.complex64)
    go = oracle_mod.irfft3(F32, n)
    return {"f": f32, "Fo": Fo, "F32": F32, "go": go}


def _pair_on_gpu(fk, dtype, d):
    n = N_FFT
    plan = fk.fftk_plan_create(n, n, n, dtype)
    try:
        x = _dev_real(d["f"])
        F = empty_c64((n, n, n // 2 + 1))
        fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, stream())
        fk.fftk_sync(plan, stream())
        del x
        Fg = _c64_to_host(F)
        Fin = _dev_c64(d["F32"])
        y = empty_real((n, n, n))
        fk.fftk_c2r(plan, Fin.data_ptr(), y.data_ptr(), 1, stream())
        fk.fftk_sync(plan, stream())
        del Fin, F
        yg = y.cpu().numpy()
    finally:
        fk.fftk_plan_destroy(plan)
    return Fg, yg


def test_pair_1024_fp32_every_element_matches_oracle(fk, pair1024):
    Fg, yg = _pair_on_gpu(fk, fk.FFTK_R32, pair1024)
    rel_f, mx_f = _compare(Fg, pair1024["Fo"])
    del Fg
    rel_i, mx_i = _compare(yg, pair1024["go"])
    print(f"\nMEASURED fft1024 fp32 r2c rel_l2 {rel_f:.3e} max/max {mx_f:.3e}; "
          f"c2r rel_l2 {rel_i:.3e} max/max {mx_i:.3e}")
    assert rel_f <= 2e-6 and mx_f <= 1e-5
    assert rel_i <= 2e-6 and mx_i <= 1e-5


def test_pair_1024_split16_every_element_matches_oracle(fk, pair1024):
    Fg, yg = _pair_on_gpu(fk, fk.FFTK_R32_SPLIT16, pair1024)
    rel_f, mx_f = _compare(Fg, pair1024["Fo"])
    del Fg
    rel_i, mx_i = _compare(yg, pair1024["go"])
    print(f"\nMEASURED fft1024 split16 r2c rel_l2 {rel_f:.3e} max/max {mx_f:.3e}; "
          f"c2r rel_l2 {rel_i:.3e} max/max {mx_i:.3e}")
    assert rel_f <= 1e-5
    assert rel_i <= 1e-5


def test_release_pair1024(pair1024):
    # the 1024^3 arrays are not needed below: free ~26 GB of host memory
    pair1024.clear()


# ------------------------------------------------------ right-hand sides ---
def _kvec(n):
    a = np.arange(n)
    k = np.where(2 * a < n, a, a - n)
    return np.meshgrid(k, k, np.arange(n // 2 + 1), indexing="ij")


def _kept(n):
    KX, KY, KZ = _kvec(n)
    return (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * np.abs(KZ) < n)


def _rhs_on_gpu(fk, dtype, u, feps):
    n = u.shape[1]
    plan = fk.fftk_plan_create(n, n, n, dtype)
    try:
        ud = _dev_c64(u)
        nd = empty_c64(u.shape)
        fk.tarang_ns_rhs(plan, ud.data_ptr(), nd.data_ptr(), fk.make_params(0.0, 0.0, feps, (1, 4)), stream())
        fk.fftk_sync(plan, stream())
        del ud
        return _c64_to_host(nd)
    finally:
        fk.fftk_plan_destroy(plan)


@pytest.fixture(scope="module")
def rhs512(oracle_mod):
    """The 512^3 decaying-turbulence initial field (k0 = 4, E = 0.5, seed 0)
    rounded to complex64, and the oracle's right-hand sides of it without and
    with constant-power forcing (eps = 0.1 on 1 <= |k|^2 <= 4)."""
    n = 512
    u = oracle_mod.ic_random(synth.normal_fields(0, 3, (n, n, n)), k0=4.0, E0=0.5).astype(np.complex64)
    uw = u.astype(np.complex128)
    No = oracle_mod.ns_rhs(uw)
    Nf = oracle_mod.ns_rhs(uw, force_eps=0.1, force_k2=(1, 4))
    return {"u": u, "No": No, "Nf": Nf}


@pytest.mark.parametrize("mode", ["fp32", "split16"])
def test_rhs_512_every_mode_matches_oracle(fk, rhs512, mode):
    dtype = fk.FFTK_R32 if mode == "fp32" else fk.FFTK_R32_SPLIT16
    tol = 1e-5 if mode == "fp32" else 3e-5
    n = 512
    for key, feps in (("No", 0.0), ("Nf", 0.1)):
        Ng = _rhs_on_gpu(fk, dtype, rhs512["u"], feps)
        rel, mx = _compare(Ng, rhs512[key])
        print(f"\nMEASURED rhs512 {mode} forcing={feps} rel_l2 {rel:.3e} max/max {mx:.3e}")
        assert rel <= tol
        # modes outside the 2/3 set are exact zeros
        kept = _kept(n)
        for c in range(3):
            assert not np.any(Ng[c][~kept])


def _embed(u, N):
    """A half spectrum [3][n][n][n/2+1] whose x and y Nyquist rows are zero,
    placed at the same wavenumbers of an N^3 grid (N >= n)."""
    n = u.shape[1]
    a = np.arange(n)
    a = a[2 * a != n]
    big = np.where(2 * a < n, a, a - n + N)
    out = np.zeros((3, N, N, N // 2 + 1), dtype=u.dtype)
    for c in range(3):
        out[c][np.ix_(big, big, np.arange(n // 2 + 1))] = u[c][np.ix_(a, a, np.arange(n // 2 + 1))]
    return out


@pytest.mark.parametrize("mode", ["fp32", "split16"])
def test_rhs_1024_band_limited_matches_oracle_at_512(fk, oracle_mod, mode):
    dtype = fk.FFTK_R32 if mode == "fp32" else fk.FFTK_R32_SPLIT16
    tol = 1e-5 if mode == "fp32" else 3e-5
    # a 256^3 random-phase field (its 2/3 set is |k_i| <= 85) with a broad
    # spectrum (k0 = 32), rounded to complex64
    u256 = oracle_mod.ic_random(synth.normal_fields(1, 3, (256, 256, 256)), k0=32.0, E0=0.5).astype(np.complex64)
    u512 = _embed(u256, 512).astype(np.complex128)
    No = oracle_mod.ns_rhs(u512)
    Nfo = oracle_mod.ns_rhs(u512, force_eps=0.1, force_k2=(1, 4))
    del u512
    u1024 = _embed(u256, 1024)
    a = np.arange(512)
    big = np.where(2 * a < 512, a, a - 512 + 1024)  # the 512^3 grid's rows inside the 1024^3 one
    inside = np.zeros(1024, dtype=bool)
    inside[big] = True
    for Nref, feps in ((No, 0.0), (Nfo, 0.1)):
        Ng = _rhs_on_gpu(fk, dtype, u1024, feps)
        sub = np.stack([Ng[c][np.ix_(big, big, np.arange(257))] for c in range(3)])
        rel, mx = _compare(sub, Nref)
        # every coefficient the 512^3 grid does not hold is zero in exact arithmetic
        out_num = 0.0
        for c in range(3):
            for i in range(1024):
                row = Ng[c, i]
                if inside[i]:
                    out_num += float(np.sum(np.abs(row[~inside, :].astype(np.complex128)) ** 2))
                    out_num += float(np.sum(np.abs(row[inside, 257:].astype(np.complex128)) ** 2))
                else:
                    out_num += float(np.sum(np.abs(row.astype(np.complex128)) ** 2))
        ref_norm = float(np.sqrt(sum(np.sum(np.abs(Nref[c]) ** 2) for c in range(3))))
        rel_out = float(np.sqrt(out_num)) / ref_norm
        print(f"\nMEASURED rhs1024 band-limited {mode} forcing={feps} rel_l2 {rel:.3e} max/max {mx:.3e} "
              f"outside {rel_out:.3e}")
        assert rel <= tol
        assert rel_out <= tol
        del Ng, sub
