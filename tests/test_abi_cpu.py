"""The C ABI without a GPU: the library loads, exports every declared entry
point, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fftk.h")


@pytest.fixture(scope="module")
def fk():
    from paper_1805_07801_gb300 import build as b

    b.build()
    import paper_1805_07801_gb300 as m

    m.lib()
    return m


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:fftk|tarang)_[a-z0-9_]+)\s*\(", text)))


def _gpu_present():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["fftk_plan_create", "fftk_r2c", "fftk_c2r", "tarang_ns_rhs", "tarang_ns_step"]:
        assert required in names


def test_every_declared_symbol_is_exported(fk):
    L = ctypes.CDLL(fk.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(fk):
    for s in range(8):
        assert fk.fftk_status_string(s).startswith("FFTK_")
    assert fk.fftk_status_string(99) == "FFTK_ERR_UNKNOWN"


@pytest.mark.parametrize(
    "shape,dtype,want",
    [
        ((5, 8, 8), 0, 2),
        ((10, 8, 8), 0, 2),
        ((8, 8, 6), 0, 2),
        ((6144, 8, 12), 0, 2),
        ((8, 8, 1), 0, 2),
        ((8, 8192, 8), 0, 2),
        ((0, 8, 8), 0, 2),
        ((8, 8, 8), 7, 1),
    ],
)
def test_plan_create_rejects_before_cuda(fk, shape, dtype, want):
    out = ctypes.c_void_p(1234)
    st = fk.lib().fftk_plan_create(*shape, dtype, ctypes.byref(out))
    assert st == want
    assert out.value is None


def test_plan_create_null_out(fk):
    assert fk.lib().fftk_plan_create(8, 8, 8, 0, None) == fk.FFTK_ERR_INVALID_ARG


def test_valid_plan_without_gpu_reports_no_device(fk):
    out = ctypes.c_void_p()
    st = fk.lib().fftk_plan_create(8, 8, 8, 0, ctypes.byref(out))
    if _gpu_present():
        assert st == fk.FFTK_OK
        assert fk.lib().fftk_plan_destroy(out) == fk.FFTK_OK
    else:
        assert st == fk.FFTK_ERR_NO_DEVICE
        assert out.value is None


def test_null_plan_calls(fk):
    L = fk.lib()
    assert L.fftk_plan_destroy(None) == fk.FFTK_ERR_INVALID_ARG
    assert L.fftk_r2c(None, None, None, 1, None) == fk.FFTK_ERR_INVALID_ARG
    assert L.fftk_c2r(None, None, None, 1, None) == fk.FFTK_ERR_INVALID_ARG
    assert L.fftk_workspace_bytes(None, 1) == 0
    assert L.fftk_launch_count(None) == -1
    assert L.tarang_ns_step(None, None, None, 1, None, None) == fk.FFTK_ERR_INVALID_ARG
    assert L.tarang_ns_rhs(None, None, None, None, None) == fk.FFTK_ERR_INVALID_ARG
    assert L.tarang_diag(None, None, 0.0, None, None) == fk.FFTK_ERR_INVALID_ARG
    assert L.fftk_profile_enable(None, 1) == fk.FFTK_ERR_INVALID_ARG


def test_kernel_names(fk):
    n = fk.fftk_kernel_kinds()
    names = [fk.fftk_kernel_name(k) for k in range(n)]
    assert len(set(names)) == n
    assert fk.fftk_kernel_name(n) == ""
    assert "ns_z_product" in names


def test_null_plan_calls_of_the_later_entry_points(fk):
    L = fk.lib()
    bad = fk.FFTK_ERR_INVALID_ARG
    assert L.tarang_transfer(None, None, None, None, None) == bad
    assert L.tarang_shell_transfer(None, None, 1, None, None, None) == bad
    assert L.fftk_forward(None, None, None, None, 1, None) == bad
    assert L.fftk_inverse(None, None, None, None, 1, None) == bad
    assert L.tarang_rbc_rhs(None, 0, None, None, None) == bad
    assert L.tarang_rbc_step(None, None, None, 1, None) == bad
    assert L.tarang_rbc_transfer(None, None, None, None) == bad
    names = [fk.fftk_kernel_name(k) for k in range(fk.fftk_kernel_kinds())]
    assert "sc_fwd" in names and "sc_inv" in names


def test_mlp_mode_entry_points_check_arguments_first(fk):
    L = fk.lib()
    bad = fk.FFTK_ERR_INVALID_ARG
    assert L.tarang_mlp_loss_grad_mode(None, None, None, None, 1, None, None, fk.TARANG_ACT_FP32, None) == bad
    assert L.tarang_mlp_forward_mode(None, None, None, None, 1, fk.TARANG_ACT_BF16, None) == bad
    assert fk.TARANG_ACT_BF16 == 0 and fk.TARANG_ACT_FP32 == 1


def _struct_fields(name):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r";", text)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if decl:
            fields.append(re.findall(r"([A-Za-z_][A-Za-z0-9_]*)\s*(?:\[[^\]]*\])?\s*$", decl)[0])
    return fields


@pytest.mark.parametrize("name", ["tarang_params", "tarang_rbc_params", "tarang_sgs_model"])
def test_binding_structs_follow_the_header(fk, name):
    # the ctypes mirrors must list the C fields in the same order
    cls = getattr(fk, name)
    assert [f[0] for f in cls._fields_] == _struct_fields(name)
