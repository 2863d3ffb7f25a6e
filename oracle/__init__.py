"""ctypes wrapper around the plain FP64 C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg; the product package never imports it.
Arrays are numpy: real fields float64[..., Nx, Ny, Nz], half spectra
complex128[..., Nx, Ny, Nz//2 + 1].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C99 + OpenMP over independent lines)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            c = ctypes
            dp = c.POINTER(c.c_double)
            vp = c.c_void_p
            L.oracle_threads.argtypes = []
            L.oracle_threads.restype = c.c_int
            L.oracle_fft1d.argtypes = [vp, vp, c.c_long, c.c_int]
            L.oracle_dft1d.argtypes = [vp, vp, c.c_long, c.c_int]
            L.oracle_rfft3.argtypes = [vp, vp, c.c_int, c.c_int, c.c_int]
            L.oracle_irfft3.argtypes = [vp, vp, c.c_int, c.c_int, c.c_int]
            L.oracle_rfft3_coeff_f32.argtypes = [vp, c.c_int, c.c_int, c.c_int, c.c_int, c.c_int, c.c_int, vp]
            L.oracle_rfft3_coeff_f32.restype = None
            L.oracle_irfft3_point_c64.argtypes = [vp, c.c_int, c.c_int, c.c_int, c.c_int, c.c_int, c.c_int]
            L.oracle_irfft3_point_c64.restype = c.c_double
            L.oracle_ns_rhs.argtypes = [vp, vp, c.c_int, vp]
            L.oracle_ns_rhs_divergence.argtypes = [vp, vp, c.c_int]
            L.oracle_ns_step.argtypes = [vp, c.c_int, vp, c.c_int]
            L.oracle_ns_step_rk4.argtypes = [vp, c.c_int, vp, c.c_int]
            L.oracle_rbc_rhs.argtypes = [vp, vp, c.c_int]
            L.oracle_rbc_step.argtypes = [vp, c.c_int, c.c_double, c.c_double, c.c_double, c.c_int, c.c_int]
            L.oracle_rbc_sff_rhs.argtypes = [vp, vp, c.c_int]
            L.oracle_rbc_sff_step.argtypes = [vp, c.c_int, c.c_double, c.c_double, c.c_double, c.c_int, c.c_int]
            L.oracle_diag.argtypes = [vp, c.c_int, c.c_double, dp, dp, vp, c.c_int]
            L.oracle_transfer.argtypes = [vp, vp, c.c_int]
            L.oracle_transfer.restype = c.c_double
            L.oracle_transfer_spectrum.argtypes = [vp, vp, c.c_int, vp, c.c_int]
            L.oracle_shell_transfer.argtypes = [vp, c.c_int, c.c_int, vp, vp]
            L.oracle_sc1d.argtypes = [vp, vp, c.c_long, c.c_int, c.c_int]
            L.oracle_transform3.argtypes = [vp, vp, c.c_int, c.c_int, c.c_int, vp]
            L.oracle_itransform3.argtypes = [vp, vp, c.c_int, c.c_int, c.c_int, vp]
            L.oracle_transform3_coeff_f32.argtypes = [vp, c.c_int, c.c_int, c.c_int, vp, c.c_int, c.c_int,
                                                      c.c_int, vp]
            L.oracle_ic_taylor_green.argtypes = [vp, c.c_int]
            L.oracle_ic_abc.argtypes = [vp, c.c_int]
            L.oracle_ic_random.argtypes = [vp, vp, c.c_int, c.c_double, c.c_double]
            L.oracle_box_filter.argtypes = [vp, c.c_int, c.c_int, vp, vp]
            L.oracle_gradient.argtypes = [vp, c.c_int, vp]
            L.oracle_les_stress.argtypes = [vp, vp, c.c_int, vp]
            L.oracle_invariants.argtypes = [vp, vp]
            L.oracle_invariants.restype = None
            L.oracle_sym_eig3.argtypes = [vp, vp, vp]
            L.oracle_sym_eig3.restype = None
            L.oracle_mlp_forward.argtypes = [vp, vp, vp, c.c_int, c.c_int]
            L.oracle_mlp_loss_grad.argtypes = [vp, vp, vp, c.c_int, c.c_int, vp]
            L.oracle_mlp_loss_grad.restype = c.c_double
            L.oracle_adam.argtypes = [vp, vp, vp, vp, c.c_int, c.c_int, c.c_double, c.c_double, c.c_double, c.c_double]
            L.oracle_adam.restype = None
            L.oracle_sgs_force.argtypes = [vp, c.c_int, vp]
            L.oracle_dealias.argtypes = [vp, c.c_int, c.c_int]
            L.oracle_project.argtypes = [vp, c.c_int]
            _lib = L
    return _lib


class NSParams(ctypes.Structure):
    _fields_ = [
        ("nu", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("force_eps", ctypes.c_double),
        ("force_k2min", ctypes.c_int),
        ("force_k2max", ctypes.c_int),
    ]


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def threads() -> int:
    return int(lib().oracle_threads())


def fft1d(x, sign: int = -1) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    _check(lib().oracle_fft1d(_ptr(x), _ptr(out), x.size, sign), "fft1d")
    return out


def dft1d(x, sign: int = -1) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    _check(lib().oracle_dft1d(_ptr(x), _ptr(out), x.size, sign), "dft1d")
    return out


def rfft3(f) -> np.ndarray:
    """Forward 3D transform with the 1/(Nx Ny Nz) factor; leading axes are a batch."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    nx, ny, nz = f.shape[-3:]
    batch = f.shape[:-3]
    out = np.empty(batch + (nx, ny, nz // 2 + 1), dtype=np.complex128)
    fv = f.reshape((-1, nx, ny, nz))
    ov = out.reshape((-1, nx, ny, nz // 2 + 1))
    for b in range(fv.shape[0]):
        _check(lib().oracle_rfft3(_ptr(fv[b]), _ptr(ov[b]), nx, ny, nz), "rfft3")
    return out


def irfft3(F, nz: int) -> np.ndarray:
    """Inverse 3D transform (no factor); `nz` is the real length of the last axis."""
    F = np.ascontiguousarray(F, dtype=np.complex128)
    nx, ny, hz = F.shape[-3:]
    if hz != nz // 2 + 1:
        raise ValueError("last axis must hold nz//2 + 1 modes")
    batch = F.shape[:-3]
    out = np.empty(batch + (nx, ny, nz), dtype=np.float64)
    Fv = F.reshape((-1, nx, ny, hz))
    ov = out.reshape((-1, nx, ny, nz))
    for b in range(Fv.shape[0]):
        _check(lib().oracle_irfft3(_ptr(Fv[b]), _ptr(ov[b]), nx, ny, nz), "irfft3")
    return out


def rfft3_coeff(f32: np.ndarray, a: int, b: int, c: int) -> complex:
    """One forward coefficient (index a, b, c) by the direct O(N^3) sum; float32 input."""
    f32 = np.ascontiguousarray(f32, dtype=np.float32)
    nx, ny, nz = f32.shape
    r = np.zeros(2, dtype=np.float64)
    lib().oracle_rfft3_coeff_f32(_ptr(f32), nx, ny, nz, a, b, c, _ptr(r))
    return complex(r[0], r[1])


def irfft3_point(F64: np.ndarray, nz: int, i: int, j: int, l: int) -> float:
    """One inverse output point by the direct sum over the half spectrum; complex64 input."""
    F64 = np.ascontiguousarray(F64, dtype=np.complex64)
    nx, ny, hz = F64.shape
    if hz != nz // 2 + 1:
        raise ValueError("last axis must hold nz//2 + 1 modes")
    return float(lib().oracle_irfft3_point_c64(_ptr(F64), nx, ny, nz, i, j, l))


def _params(nu=0.0, dt=0.0, force_eps=0.0, force_k2=(1, 4)) -> NSParams:
    return NSParams(nu, dt, force_eps, int(force_k2[0]), int(force_k2[1]))


def ns_rhs(uhat, nu=0.0, dt=0.0, force_eps=0.0, force_k2=(1, 4)) -> np.ndarray:
    uhat = np.ascontiguousarray(uhat, dtype=np.complex128)
    n = uhat.shape[1]
    out = np.empty_like(uhat)
    p = _params(nu, dt, force_eps, force_k2)
    _check(lib().oracle_ns_rhs(_ptr(uhat), _ptr(out), n, ctypes.byref(p)), "ns_rhs")
    return out


def ns_rhs_divergence(uhat) -> np.ndarray:
    uhat = np.ascontiguousarray(uhat, dtype=np.complex128)
    out = np.empty_like(uhat)
    _check(lib().oracle_ns_rhs_divergence(_ptr(uhat), _ptr(out), uhat.shape[1]), "ns_rhs_divergence")
    return out


def ns_step(uhat, nu, dt, nsteps=1, force_eps=0.0, force_k2=(1, 4)) -> np.ndarray:
    u = np.array(uhat, dtype=np.complex128, order="C", copy=True)
    p = _params(nu, dt, force_eps, force_k2)
    _check(lib().oracle_ns_step(_ptr(u), u.shape[1], ctypes.byref(p), nsteps), "ns_step")
    return u


FOURIER, SINE, COSINE = 0, 1, 2
_BASIS = {"F": FOURIER, "S": SINE, "C": COSINE}


def _kinds(basis) -> np.ndarray:
    if isinstance(basis, str):
        basis = [_BASIS[ch] for ch in basis]
    return np.ascontiguousarray(basis, dtype=np.int32)


def sc1d(x, kind, direction) -> np.ndarray:
    """Sine (kind 'S') or cosine ('C') transform of a line; direction -1 forward, +1 inverse."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    _check(lib().oracle_sc1d(_ptr(x), _ptr(out), x.size, _BASIS[kind], direction), "sc1d")
    return out


def transform3(f, basis) -> np.ndarray:
    """Forward 3D transform with a basis per axis, e.g. 'SFF' (x sine, y and z Fourier)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    nx, ny, nz = f.shape
    k = _kinds(basis)
    hz = nz // 2 + 1 if k[2] == FOURIER else nz
    out = np.empty((nx, ny, hz), dtype=np.complex128)
    _check(lib().oracle_transform3(_ptr(f), _ptr(out), nx, ny, nz, _ptr(k)), "transform3")
    return out


def itransform3(F, nz: int, basis) -> np.ndarray:
    F = np.ascontiguousarray(F, dtype=np.complex128)
    nx, ny = F.shape[0], F.shape[1]
    k = _kinds(basis)
    out = np.empty((nx, ny, nz), dtype=np.float64)
    _check(lib().oracle_itransform3(_ptr(F), _ptr(out), nx, ny, nz, _ptr(k)), "itransform3")
    return out


def transform3_coeff(f32: np.ndarray, basis, a: int, b: int, c: int) -> complex:
    """Coefficient (a, b, c) of transform3 of an FP32 field, by its definition."""
    f32 = np.ascontiguousarray(f32, dtype=np.float32)
    nx, ny, nz = f32.shape
    k = _kinds(basis)
    out = np.zeros(2, dtype=np.float64)
    _check(lib().oracle_transform3_coeff_f32(_ptr(f32), nx, ny, nz, _ptr(k), a, b, c, _ptr(out)),
           "transform3_coeff")
    return complex(out[0], out[1])


def ns_step_rk4(uhat, nu, dt, nsteps=1, force_eps=0.0, force_k2=(1, 4)) -> np.ndarray:
    u = np.array(uhat, dtype=np.complex128, order="C", copy=True)
    p = _params(nu, dt, force_eps, force_k2)
    _check(lib().oracle_ns_step_rk4(_ptr(u), u.shape[1], ctypes.byref(p), nsteps), "ns_step_rk4")
    return u


def rbc_rhs(state) -> np.ndarray:
    """(N_u, N_theta) of a Rayleigh-Benard state [4][n][n][n/2+1]."""
    st = np.ascontiguousarray(state, dtype=np.complex128)
    out = np.empty_like(st)
    _check(lib().oracle_rbc_rhs(_ptr(st), _ptr(out), st.shape[1]), "rbc_rhs")
    return out


def rbc_step(state, Ra, Pr, dt, nsteps=1, scheme=1) -> np.ndarray:
    st = np.array(state, dtype=np.complex128, order="C", copy=True)
    _check(lib().oracle_rbc_step(_ptr(st), st.shape[1], float(Ra), float(Pr), float(dt), nsteps, scheme),
           "rbc_step")
    return st


def rbc_sff_rhs(state) -> np.ndarray:
    """(N_u, N_theta) between free-slip plates: u_x, theta sine along x, u_y, u_z cosine."""
    st = np.ascontiguousarray(state, dtype=np.complex128)
    out = np.empty_like(st)
    _check(lib().oracle_rbc_sff_rhs(_ptr(st), _ptr(out), st.shape[1]), "rbc_sff_rhs")
    return out


def rbc_sff_step(state, Ra, Pr, dt, nsteps=1, scheme=1) -> np.ndarray:
    st = np.array(state, dtype=np.complex128, order="C", copy=True)
    _check(lib().oracle_rbc_sff_step(_ptr(st), st.shape[1], float(Ra), float(Pr), float(dt), nsteps, scheme),
           "rbc_sff_step")
    return st


def kmax_shell(n: int) -> int:
    return int(np.floor(np.sqrt(3.0) * (n // 2) + 0.5)) + 1


def diag(uhat, nu=0.0, kmax=None):
    """Returns (E, eps, E(K) for K = 0..kmax)."""
    uhat = np.ascontiguousarray(uhat, dtype=np.complex128)
    n = uhat.shape[1]
    kmax = kmax_shell(n) if kmax is None else kmax
    E = ctypes.c_double()
    eps = ctypes.c_double()
    EK = np.zeros(kmax + 1, dtype=np.float64)
    _check(lib().oracle_diag(_ptr(uhat), n, nu, ctypes.byref(E), ctypes.byref(eps), _ptr(EK), kmax), "diag")
    return E.value, eps.value, EK


def transfer(uhat, nhat) -> float:
    uhat = np.ascontiguousarray(uhat, dtype=np.complex128)
    nhat = np.ascontiguousarray(nhat, dtype=np.complex128)
    return float(lib().oracle_transfer(_ptr(uhat), _ptr(nhat), uhat.shape[1]))


def transfer_spectrum(uhat, nhat, kmax=None) -> np.ndarray:
    """T(K) = sum over shell K of w Re(conj(u) . N), K = 0..kmax."""
    uhat = np.ascontiguousarray(uhat, dtype=np.complex128)
    nhat = np.ascontiguousarray(nhat, dtype=np.complex128)
    n = uhat.shape[1]
    kmax = kmax_shell(n) if kmax is None else kmax
    T = np.zeros(kmax + 1, dtype=np.float64)
    _check(lib().oracle_transfer_spectrum(_ptr(uhat), _ptr(nhat), n, _ptr(T), kmax), "transfer_spectrum")
    return T


def shell_transfer(uhat, bounds) -> np.ndarray:
    """T[r, g]: energy rate from shell g to shell r, shells bounds[i] <= nint|k| < bounds[i+1]."""
    uhat = np.ascontiguousarray(uhat, dtype=np.complex128)
    b = np.ascontiguousarray(bounds, dtype=np.int32)
    S = len(b) - 1
    T = np.zeros((S, S), dtype=np.float64)
    _check(lib().oracle_shell_transfer(_ptr(uhat), uhat.shape[1], S, _ptr(b), _ptr(T)), "shell_transfer")
    return T


def ic_taylor_green(n: int) -> np.ndarray:
    u = np.empty((3, n, n, n // 2 + 1), dtype=np.complex128)
    _check(lib().oracle_ic_taylor_green(_ptr(u), n), "ic_taylor_green")
    return u


def ic_abc(n: int) -> np.ndarray:
    u = np.empty((3, n, n, n // 2 + 1), dtype=np.complex128)
    _check(lib().oracle_ic_abc(_ptr(u), n), "ic_abc")
    return u


def ic_random(normals, k0=4.0, E0=0.5) -> np.ndarray:
    normals = np.ascontiguousarray(normals, dtype=np.float64)
    n = normals.shape[1]
    u = np.empty((3, n, n, n // 2 + 1), dtype=np.complex128)
    _check(lib().oracle_ic_random(_ptr(normals), _ptr(u), n, k0, E0), "ic_random")
    return u


def dealias(F, nfields=None):
    F = np.array(F, dtype=np.complex128, order="C", copy=True)
    n = F.shape[-2]
    nf = nfields if nfields is not None else (F.size // (n * n * (n // 2 + 1)))
    _check(lib().oracle_dealias(_ptr(F), nf, n), "dealias")
    return F


def project(uhat):
    u = np.array(uhat, dtype=np.complex128, order="C", copy=True)
    _check(lib().oracle_project(_ptr(u), u.shape[1]), "project")
    return u


# ------------------------------------------------------------------ closure --
MLP_NPARAMS = 9094
MLP_DIMS = (5, 64, 64, 64, 6)


def box_filter(u, factor):
    """u: real [3][n][n][n] -> (ubar [3][m]^3, tau [6][m]^3 in order xx, yy, zz, xy, xz, yz)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = u.shape[1]
    m = n // factor
    ubar = np.empty((3, m, m, m))
    tau = np.empty((6, m, m, m))
    _check(lib().oracle_box_filter(_ptr(u), n, factor, _ptr(ubar), _ptr(tau)), "box_filter")
    return ubar, tau


def les_stress(ubar, tau):
    """T[tau + ubar_i ubar_j - (T ubar)_i (T ubar)_j] on the coarse grid (T: the 2/3 truncation)."""
    ubar = np.ascontiguousarray(ubar, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    m = ubar.shape[1]
    out = np.empty((6, m, m, m))
    _check(lib().oracle_les_stress(_ptr(ubar), _ptr(tau), m, _ptr(out)), "les_stress")
    return out


def gradient(u):
    """A[i*3+j] = d u_i / d x_j of a real [3][m]^3 field from its 2/3-truncated spectrum."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    m = u.shape[1]
    A = np.empty((9, m, m, m))
    _check(lib().oracle_gradient(_ptr(u), m, _ptr(A)), "gradient")
    return A


def invariants(A9):
    A9 = np.ascontiguousarray(A9, dtype=np.float64)
    out = np.empty(5)
    lib().oracle_invariants(_ptr(A9), _ptr(out))
    return out


def sym_eig3(S9):
    S9 = np.ascontiguousarray(S9, dtype=np.float64)
    lam = np.empty(3)
    Q = np.empty(9)
    lib().oracle_sym_eig3(_ptr(S9), _ptr(lam), _ptr(Q))
    return lam, Q.reshape(3, 3)


def mlp_forward(params, x, bf16_acts=True):
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    B = x.shape[0]
    y = np.empty((B, 6))
    _check(lib().oracle_mlp_forward(_ptr(params), _ptr(x), _ptr(y), B, int(bf16_acts)), "mlp_forward")
    return y


def mlp_loss_grad(params, x, t, bf16_acts=True):
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    g = np.empty(MLP_NPARAMS)
    loss = lib().oracle_mlp_loss_grad(_ptr(params), _ptr(x), _ptr(t), x.shape[0], int(bf16_acts), _ptr(g))
    return float(loss), g


def adam(params, m, v, grad, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on params, m, v (float64 arrays)."""
    grad = np.ascontiguousarray(grad, dtype=np.float64)
    lib().oracle_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), params.size, step, lr, beta1, beta2, eps)


def sgs_force(tau):
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    n = tau.shape[1]
    f = np.empty((3, n, n, n // 2 + 1), dtype=np.complex128)
    _check(lib().oracle_sgs_force(_ptr(tau), n, _ptr(f)), "sgs_force")
    return f
