"""Python binding of libfftk (GB300 FFTK/Tarang hot path).

Argument marshalling only: every function here forwards to the C ABI declared
in include/fftk.h (same names); all arithmetic runs in the library's CUDA
kernels.  Device buffers are passed as integer addresses (e.g. a torch CUDA
tensor's data_ptr()) and streams as integer cudaStream_t handles
(torch.cuda.current_stream().cuda_stream).  The library must be built
(build.build()); there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfftk.so")

FFTK_OK = 0
FFTK_ERR_INVALID_ARG = 1
FFTK_ERR_UNSUPPORTED_SIZE = 2
FFTK_ERR_NO_DEVICE = 3
FFTK_ERR_OOM = 4
FFTK_ERR_CUDA = 5
FFTK_ERR_NONFINITE = 6
FFTK_ERR_TIMEOUT = 7

FFTK_R32 = 0
FFTK_R32_SPLIT16 = 1


class FFTKError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {fftk_status_string(status)} ({status})"
        if status in (FFTK_ERR_NO_DEVICE, FFTK_ERR_OOM, FFTK_ERR_CUDA):
            cause = lib().fftk_last_cuda_error().decode()
            if cause:
                msg += f" [{cause}]"
        super().__init__(msg)


class tarang_sgs_model(ctypes.Structure):
    _fields_ = [
        ("params", ctypes.c_void_p),
        ("in_shift", ctypes.c_float * 5),
        ("in_scale", ctypes.c_float * 5),
        ("out_scale", ctypes.c_float * 6),
    ]


class tarang_params(ctypes.Structure):
    _fields_ = [
        ("nu", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("force_eps", ctypes.c_double),
        ("force_k2min", ctypes.c_int),
        ("force_k2max", ctypes.c_int),
        ("sgs_model", ctypes.POINTER(tarang_sgs_model)),
        ("scheme", ctypes.c_int),
    ]


TARANG_RK2, TARANG_RK4 = 0, 1
TARANG_RBC_FFF, TARANG_RBC_SFF = 0, 1


class tarang_rbc_params(ctypes.Structure):
    _fields_ = [
        ("Ra", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("scheme", ctypes.c_int),
        ("basis", ctypes.c_int),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libfftk.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1805_07801_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        c = ctypes
        vp, i, d, ll = c.c_void_p, c.c_int, c.c_double, c.c_longlong
        sig = {
            "fftk_status_string": ([i], c.c_char_p),
            "fftk_last_cuda_error": ([], c.c_char_p),
            "fftk_plan_create": ([i, i, i, i, c.POINTER(vp)], i),
            "fftk_plan_destroy": ([vp], i),
            "fftk_workspace_bytes": ([vp, i], c.c_size_t),
            "fftk_set_workspace": ([vp, vp, c.c_size_t], i),
            "fftk_r2c": ([vp, vp, vp, i, vp], i),
            "fftk_c2r": ([vp, vp, vp, i, vp], i),
            "tarang_ns_rhs": ([vp, vp, vp, c.POINTER(tarang_params), vp], i),
            "tarang_ns_step": ([vp, vp, c.POINTER(tarang_params), i, vp, vp], i),
            "tarang_diag_kmax": ([vp], i),
            "tarang_diag": ([vp, vp, d, vp, vp], i),
            "tarang_diag_noalloc": ([i, vp, d, vp, vp], i),
            "tarang_rbc_rhs": ([vp, i, vp, vp, vp], i),
            "tarang_rbc_transfer": ([vp, vp, vp, vp], i),
            "tarang_rbc_step": ([vp, vp, c.POINTER(tarang_rbc_params), i, vp], i),
            "fftk_forward": ([vp, vp, vp, vp, i, vp], i),
            "fftk_inverse": ([vp, vp, vp, vp, i, vp], i),
            "tarang_transfer": ([vp, vp, c.POINTER(tarang_params), vp, vp], i),
            "tarang_shell_transfer": ([vp, vp, i, vp, vp, vp], i),
            "tarang_ic_random": ([vp, vp, vp, d, d, vp], i),
            "tarang_dealias_project": ([vp, vp, vp], i),
            "fftk_fill_normal": ([vp, ll, i, i, vp], i),
            "fftk_fill_uniform": ([vp, ll, i, i, vp], i),
            "fftk_sync": ([vp, vp], i),
            "tarang_box_filter": ([vp, vp, i, vp, vp, vp], i),
            "tarang_closure_features": ([vp, vp, vp, vp, vp, vp, vp], i),
            "tarang_mlp_create": ([i, c.POINTER(vp)], i),
            "tarang_mlp_destroy": ([vp], i),
            "tarang_mlp_forward": ([vp, vp, vp, vp, i, vp], i),
            "tarang_mlp_sync": ([vp, vp], i),
            "tarang_sgs_train": ([vp, vp, vp, vp, i, i, vp, vp, ll, i, c.c_float, c.c_ulonglong, vp, i, vp], i),
            "tarang_mlp_loss_grad": ([vp, vp, vp, vp, i, vp, vp, vp], i),
            "tarang_les_stress": ([vp, vp, vp, vp, vp], i),
            "tarang_mlp_loss_grad_mode": ([vp, vp, vp, vp, i, vp, vp, i, vp], i),
            "tarang_mlp_forward_mode": ([vp, vp, vp, vp, i, i, vp], i),
            "tarang_mlp_adam": ([vp, vp, vp, vp, i, c.c_float, c.c_float, c.c_float, c.c_float, vp], i),
            "tarang_mlp_train_step": ([vp, vp, vp, vp, i, vp, vp, i, c.c_float, vp, vp], i),
            "fftk_launch_count": ([vp], ll),
            "fftk_profile_enable": ([vp, i], i),
            "fftk_profile_read": ([vp, i, c.POINTER(d), c.POINTER(ll)], i),
            "fftk_kernel_kinds": ([], i),
            "fftk_kernel_name": ([i], c.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _vp(x):
    return ctypes.c_void_p(int(x) if x is not None else 0)


def _check(st: int, where: str):
    if st != FFTK_OK:
        raise FFTKError(st, where)


def fftk_status_string(s: int) -> str:
    return lib().fftk_status_string(int(s)).decode()


def fftk_plan_create(nx: int, ny: int, nz: int, dtype: int = FFTK_R32) -> int:
    out = ctypes.c_void_p()
    _check(lib().fftk_plan_create(nx, ny, nz, dtype, ctypes.byref(out)), "fftk_plan_create")
    return out.value


def fftk_plan_destroy(plan: int) -> None:
    _check(lib().fftk_plan_destroy(_vp(plan)), "fftk_plan_destroy")


def fftk_workspace_bytes(plan: int, batch: int) -> int:
    return int(lib().fftk_workspace_bytes(_vp(plan), batch))


def fftk_set_workspace(plan: int, dev_ptr, nbytes: int) -> None:
    _check(lib().fftk_set_workspace(_vp(plan), _vp(dev_ptr), nbytes), "fftk_set_workspace")


def fftk_r2c(plan: int, in_ptr, out_ptr, batch: int = 1, stream=0) -> None:
    _check(lib().fftk_r2c(_vp(plan), _vp(in_ptr), _vp(out_ptr), batch, _vp(stream)), "fftk_r2c")


def fftk_c2r(plan: int, in_ptr, out_ptr, batch: int = 1, stream=0) -> None:
    _check(lib().fftk_c2r(_vp(plan), _vp(in_ptr), _vp(out_ptr), batch, _vp(stream)), "fftk_c2r")


def make_params(nu: float, dt: float = 0.0, force_eps: float = 0.0, force_k2=(1, 4), sgs_model=None,
                scheme: int = TARANG_RK2) -> tarang_params:
    p = tarang_params(float(nu), float(dt), float(force_eps), int(force_k2[0]), int(force_k2[1]))
    p.scheme = int(scheme)
    if sgs_model is not None:
        p.sgs_model = ctypes.pointer(sgs_model)
        p._model_ref = sgs_model  # keep alive with the params
    return p


def make_sgs_model(params_ptr, in_shift, in_scale, out_scale) -> tarang_sgs_model:
    m = tarang_sgs_model()
    m.params = int(params_ptr)
    for i in range(5):
        m.in_shift[i] = float(in_shift[i])
        m.in_scale[i] = float(in_scale[i])
    for i in range(6):
        m.out_scale[i] = float(out_scale[i])
    return m


def tarang_ns_rhs(plan: int, uhat_ptr, nhat_ptr, params: tarang_params, stream=0) -> None:
    _check(lib().tarang_ns_rhs(_vp(plan), _vp(uhat_ptr), _vp(nhat_ptr), ctypes.byref(params), _vp(stream)),
           "tarang_ns_rhs")


def tarang_diag_kmax(plan: int) -> int:
    return int(lib().tarang_diag_kmax(_vp(plan)))


def tarang_ns_step(plan: int, uhat_ptr, params: tarang_params, nsteps: int = 1, diag: bool = False, stream=0):
    """Advance nsteps; with diag=True returns (E, eps, E(K) list)."""
    buf = None
    if diag:
        buf = (ctypes.c_double * (2 + tarang_diag_kmax(plan) + 1))()
    _check(lib().tarang_ns_step(_vp(plan), _vp(uhat_ptr), ctypes.byref(params), nsteps,
                                ctypes.cast(buf, ctypes.c_void_p) if buf is not None else None, _vp(stream)),
           "tarang_ns_step")
    if buf is None:
        return None
    vals = list(buf)
    return vals[0], vals[1], vals[2:]


def tarang_rbc_rhs(plan: int, state_ptr, out_ptr, stream=0, basis: int = TARANG_RBC_FFF) -> None:
    _check(lib().tarang_rbc_rhs(_vp(plan), int(basis), _vp(state_ptr), _vp(out_ptr), _vp(stream)),
           "tarang_rbc_rhs")


def tarang_rbc_step(plan: int, state_ptr, Ra: float, Pr: float, dt: float, nsteps: int = 1,
                    scheme: int = TARANG_RK4, stream=0, basis: int = TARANG_RBC_FFF) -> None:
    prm = tarang_rbc_params(float(Ra), float(Pr), float(dt), int(scheme), int(basis))
    _check(lib().tarang_rbc_step(_vp(plan), _vp(state_ptr), ctypes.byref(prm), int(nsteps), _vp(stream)),
           "tarang_rbc_step")


def tarang_rbc_transfer(plan: int, state_ptr, stream=0):
    """((sum T_u, T_u list, Pi_u list), (sum T_theta, T_theta list, Pi_theta list)); synchronises."""
    nb = tarang_diag_kmax(plan) + 1
    buf = (ctypes.c_double * (2 * (1 + 2 * nb)))()
    _check(lib().tarang_rbc_transfer(_vp(plan), _vp(state_ptr), ctypes.cast(buf, ctypes.c_void_p), _vp(stream)),
           "tarang_rbc_transfer")
    v = list(buf)
    h = 1 + 2 * nb
    return tuple((v[o], v[o + 1:o + 1 + nb], v[o + 1 + nb:o + h]) for o in (0, h))


FFTK_FOURIER, FFTK_SINE, FFTK_COSINE = 0, 1, 2
_BASIS_CHARS = {"F": FFTK_FOURIER, "S": FFTK_SINE, "C": FFTK_COSINE}


def _basis(basis):
    if isinstance(basis, str):
        basis = [_BASIS_CHARS[ch] for ch in basis]
    return (ctypes.c_int * 3)(*[int(b) for b in basis])


def fftk_forward(plan: int, basis, in_ptr, out_ptr, batch: int = 1, stream=0) -> None:
    """Forward transform with a basis per axis ('SFF', 'CCS', ... or three fftk_basis codes)."""
    b = _basis(basis)
    _check(lib().fftk_forward(_vp(plan), ctypes.cast(b, ctypes.c_void_p), _vp(in_ptr), _vp(out_ptr), batch,
                              _vp(stream)), "fftk_forward")


def fftk_inverse(plan: int, basis, in_ptr, out_ptr, batch: int = 1, stream=0) -> None:
    b = _basis(basis)
    _check(lib().fftk_inverse(_vp(plan), ctypes.cast(b, ctypes.c_void_p), _vp(in_ptr), _vp(out_ptr), batch,
                              _vp(stream)), "fftk_inverse")


def tarang_transfer(plan: int, uhat_ptr, params: tarang_params = None, stream=0):
    """(sum_K T(K), T(K) list, Pi(K) list) of a velocity state; synchronises."""
    nb = tarang_diag_kmax(plan) + 1
    buf = (ctypes.c_double * (1 + 2 * nb))()
    _check(lib().tarang_transfer(_vp(plan), _vp(uhat_ptr), ctypes.byref(params) if params is not None else None,
                                 ctypes.cast(buf, ctypes.c_void_p), _vp(stream)), "tarang_transfer")
    vals = list(buf)
    return vals[0], vals[1:1 + nb], vals[1 + nb:]


def tarang_shell_transfer(plan: int, uhat_ptr, bounds, stream=0):
    """Shell-to-shell transfer matrix T[r][g] (list of rows) for the shells
    bounds[i] <= nint|k| < bounds[i+1]; synchronises."""
    S = len(bounds) - 1
    b = (ctypes.c_int * len(bounds))(*[int(v) for v in bounds])
    buf = (ctypes.c_double * max(S * S, 1))()
    _check(lib().tarang_shell_transfer(_vp(plan), _vp(uhat_ptr), S, ctypes.cast(b, ctypes.c_void_p),
                                       ctypes.cast(buf, ctypes.c_void_p), _vp(stream)), "tarang_shell_transfer")
    vals = list(buf)
    return [vals[r * S:(r + 1) * S] for r in range(S)]


def tarang_diag(plan: int, uhat_ptr, nu: float, stream=0):
    """(E, eps, E(K) list) of a velocity state; synchronises."""
    buf = (ctypes.c_double * (2 + tarang_diag_kmax(plan) + 1))()
    _check(lib().tarang_diag(_vp(plan), _vp(uhat_ptr), float(nu), ctypes.cast(buf, ctypes.c_void_p), _vp(stream)),
           "tarang_diag")
    vals = list(buf)
    return vals[0], vals[1], vals[2:]


def tarang_diag_noalloc(n: int, uhat_ptr, nu: float, diag_dev_ptr, stream=0) -> None:
    """Diagnostics into a caller-owned device buffer of 2 + kmax + 1 doubles; allocates nothing."""
    _check(lib().tarang_diag_noalloc(int(n), _vp(uhat_ptr), float(nu), _vp(diag_dev_ptr), _vp(stream)),
           "tarang_diag_noalloc")


def tarang_ic_random(plan: int, normals_ptr, uhat_ptr, k0: float = 4.0, E0: float = 0.5, stream=0) -> None:
    _check(lib().tarang_ic_random(_vp(plan), _vp(normals_ptr), _vp(uhat_ptr), float(k0), float(E0), _vp(stream)),
           "tarang_ic_random")


def tarang_dealias_project(plan: int, uhat_ptr, stream=0) -> None:
    _check(lib().tarang_dealias_project(_vp(plan), _vp(uhat_ptr), _vp(stream)), "tarang_dealias_project")


def fftk_fill_normal(dev_ptr, count: int, seed: int, field: int, stream=0) -> None:
    _check(lib().fftk_fill_normal(_vp(dev_ptr), int(count), int(seed), int(field), _vp(stream)), "fftk_fill_normal")


def fftk_fill_uniform(dev_ptr, count: int, seed: int, field: int, stream=0) -> None:
    _check(lib().fftk_fill_uniform(_vp(dev_ptr), int(count), int(seed), int(field), _vp(stream)),
           "fftk_fill_uniform")


def tarang_box_filter(plan: int, uhat_ptr, factor: int, ubar_ptr, tau_ptr, stream=0) -> None:
    _check(lib().tarang_box_filter(_vp(plan), _vp(uhat_ptr), int(factor), _vp(ubar_ptr), _vp(tau_ptr), _vp(stream)),
           "tarang_box_filter")


def tarang_closure_features(plan: int, ubar_ptr, tau_ptr, inv_ptr, frame_ptr, tau_frame_ptr, stream=0) -> None:
    _check(lib().tarang_closure_features(_vp(plan), _vp(ubar_ptr), _vp(tau_ptr), _vp(inv_ptr), _vp(frame_ptr),
                                         _vp(tau_frame_ptr), _vp(stream)), "tarang_closure_features")


def tarang_les_stress(plan: int, ubar_ptr, tau_ptr, out_ptr, stream=0) -> None:
    _check(lib().tarang_les_stress(_vp(plan), _vp(ubar_ptr), _vp(tau_ptr), _vp(out_ptr), _vp(stream)),
           "tarang_les_stress")


def tarang_mlp_create(max_batch: int) -> int:
    out = ctypes.c_void_p()
    _check(lib().tarang_mlp_create(int(max_batch), ctypes.byref(out)), "tarang_mlp_create")
    return out.value


def tarang_mlp_destroy(m: int) -> None:
    _check(lib().tarang_mlp_destroy(_vp(m)), "tarang_mlp_destroy")


def tarang_mlp_forward(m: int, params_ptr, x_ptr, y_ptr, B: int, stream=0) -> None:
    _check(lib().tarang_mlp_forward(_vp(m), _vp(params_ptr), _vp(x_ptr), _vp(y_ptr), int(B), _vp(stream)),
           "tarang_mlp_forward")


def tarang_sgs_train(m: int, params_ptr, m_ptr, v_ptr, first_step: int, steps: int, x_ptr, t_ptr, nsamples: int,
                     batch: int, lr: float, seed: int, loss_log_ptr=0, log_every: int = 1, stream=0) -> None:
    _check(lib().tarang_sgs_train(_vp(m), _vp(params_ptr), _vp(m_ptr), _vp(v_ptr), int(first_step), int(steps),
                                  _vp(x_ptr), _vp(t_ptr), int(nsamples), int(batch), float(lr),
                                  ctypes.c_ulonglong(int(seed)), _vp(loss_log_ptr), int(log_every), _vp(stream)),
           "tarang_sgs_train")


def tarang_mlp_sync(m: int, stream=0) -> None:
    _check(lib().tarang_mlp_sync(_vp(m), _vp(stream)), "tarang_mlp_sync")


def tarang_mlp_loss_grad(m: int, params_ptr, x_ptr, t_ptr, B: int, grad_ptr, loss_ptr, stream=0) -> None:
    _check(lib().tarang_mlp_loss_grad(_vp(m), _vp(params_ptr), _vp(x_ptr), _vp(t_ptr), int(B), _vp(grad_ptr),
                                      _vp(loss_ptr), _vp(stream)), "tarang_mlp_loss_grad")


TARANG_ACT_BF16, TARANG_ACT_FP32 = 0, 1


def tarang_mlp_loss_grad_mode(m: int, params_ptr, x_ptr, t_ptr, B: int, grad_ptr, loss_ptr, act_mode: int,
                              stream=0) -> None:
    _check(lib().tarang_mlp_loss_grad_mode(_vp(m), _vp(params_ptr), _vp(x_ptr), _vp(t_ptr), int(B), _vp(grad_ptr),
                                           _vp(loss_ptr), int(act_mode), _vp(stream)), "tarang_mlp_loss_grad_mode")


def tarang_mlp_forward_mode(m: int, params_ptr, x_ptr, y_ptr, B: int, act_mode: int, stream=0) -> None:
    _check(lib().tarang_mlp_forward_mode(_vp(m), _vp(params_ptr), _vp(x_ptr), _vp(y_ptr), int(B), int(act_mode),
                                         _vp(stream)), "tarang_mlp_forward_mode")


def tarang_mlp_adam(params_ptr, m_ptr, v_ptr, grad_ptr, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                    stream=0) -> None:
    _check(lib().tarang_mlp_adam(_vp(params_ptr), _vp(m_ptr), _vp(v_ptr), _vp(grad_ptr), int(step), lr, beta1,
                                 beta2, eps, _vp(stream)), "tarang_mlp_adam")


def tarang_mlp_train_step(m: int, params_ptr, m_ptr, v_ptr, step: int, x_ptr, t_ptr, B: int, lr: float,
                          loss_ptr, stream=0) -> None:
    _check(lib().tarang_mlp_train_step(_vp(m), _vp(params_ptr), _vp(m_ptr), _vp(v_ptr), int(step), _vp(x_ptr),
                                       _vp(t_ptr), int(B), float(lr), _vp(loss_ptr), _vp(stream)),
           "tarang_mlp_train_step")


def fftk_sync(plan: int, stream=0) -> None:
    _check(lib().fftk_sync(_vp(plan), _vp(stream)), "fftk_sync")


def fftk_launch_count(plan: int) -> int:
    return int(lib().fftk_launch_count(_vp(plan)))


def fftk_profile_enable(plan: int, on: bool = True) -> None:
    _check(lib().fftk_profile_enable(_vp(plan), int(bool(on))), "fftk_profile_enable")


def fftk_profile_read(plan: int, kind: int):
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(lib().fftk_profile_read(_vp(plan), kind, ctypes.byref(ms), ctypes.byref(n)), "fftk_profile_read")
    return ms.value, n.value


def fftk_kernel_kinds() -> int:
    return int(lib().fftk_kernel_kinds())


def fftk_kernel_name(kind: int) -> str:
    r = lib().fftk_kernel_name(kind)
    return r.decode() if r else ""


def kernel_index(name: str) -> int:
    for k in range(fftk_kernel_kinds()):
        if fftk_kernel_name(k) == name:
            return k
    raise KeyError(name)
