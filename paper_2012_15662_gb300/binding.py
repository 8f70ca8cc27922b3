"""ctypes binding of the engine's C ABI (`include/donof_ri.h`).

Argument marshalling only: every computation runs in `libdonof_ri.so`.  The
functions carry the ABI's names; arrays may be numpy FP64 arrays (host
memory) or torch FP64 CUDA tensors (device memory), both C-contiguous.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdonof_ri.so")

DONOF_RI_OK = 0
DONOF_RI_E_ARG = -1
DONOF_RI_E_OOM = -2
DONOF_RI_E_CUDA = -3
DONOF_RI_E_METRIC_NOT_PD = -4
DONOF_RI_E_NONFINITE = -5
DONOF_RI_E_TIMEOUT = -6
DONOF_RI_E_STATE = -7
DONOF_RI_E_UNSUPPORTED = -8

DONOF_RI_FP64 = 0
DONOF_RI_TF32X3 = 1
DONOF_RI_SLICE4 = 2
DONOF_RI_HALF = 0
DONOF_RI_FULL = 1

DONOF_RI_FETCH_B = 0
DONOF_RI_FETCH_BHALF = 1
DONOF_RI_FETCH_DIAG = 2
DONOF_RI_FETCH_HCORE = 3
DONOF_RI_FETCH_OVERLAP = 4
DONOF_RI_FETCH_METRIC = 5
DONOF_RI_FETCH_ENUC = 6
DONOF_RI_FETCH_OCC = 7

DONOF_RI_METRIC_CHOLESKY = 0
DONOF_RI_METRIC_MODIFIED = 1

# Names of every entry point declared in include/donof_ri.h.
EXPORTS = [
    "donof_ri_init", "donof_ri_init_ex", "donof_ri_metric_info", "donof_ri_transform", "donof_ri_jk_mo", "donof_ri_jk_ao_batch",
    "donof_ri_energy_lagrangian", "donof_ri_fetch", "donof_ri_sync", "donof_ri_destroy",
    "donof_ri_strerror", "donof_ri_launch_count", "donof_ri_profile", "donof_ri_profile_read",
    "donof_ri_iteration", "donof_ri_jmo_noalloc", "donof_ri_optimize_occupations",
    "donof_ri_on_features", "donof_ri_gamma_guess", "donof_ri_rotate_orbitals", "donof_ri_autotune", "donof_ri_set_schedule", "donof_ri_exact_jk",
    "donof_ri_energy_lagrangian_contracted", "donof_ri_flambda_step", "donof_ri_check_wait_timeout", "donof_ri_rhf", "donof_ri_apply_rotation",
    "donof_mlp_create", "donof_mlp_param_count", "donof_mlp_set_params", "donof_mlp_get_params",
    "donof_mlp_set_normalization", "donof_mlp_forward", "donof_mlp_loss_grad", "donof_mlp_train_step",
    "donof_mlp_destroy",
]

ROWS = ["half", "diag", "full_k", "j", "jao", "kao", "energy", "other"]


class DonofError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


class Options(ctypes.Structure):
    _fields_ = [("metric", ctypes.c_int), ("metric_tol", ctypes.c_double)]


class System(ctypes.Structure):
    _fields_ = [
        ("nbf", ctypes.c_int), ("naux", ctypes.c_int), ("n_atoms", ctypes.c_int),
        ("n_strong", ctypes.c_int), ("n_weak_per", ctypes.c_int),
        ("atom_xyz", ctypes.c_void_p), ("atom_charge", ctypes.c_void_p),
        ("bf_atom", ctypes.c_void_p), ("bf_alpha", ctypes.c_void_p),
        ("aux_atom", ctypes.c_void_p), ("aux_alpha", ctypes.c_void_p),
        ("subspace", ctypes.c_void_p), ("weak_rank", ctypes.c_void_p),
    ]


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libdonof_ri.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA engine first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.donof_ri_init.argtypes = [ctypes.POINTER(System), i, vp, ctypes.POINTER(vp)]
    lib.donof_ri_init_ex.argtypes = [ctypes.POINTER(System), i, vp, ctypes.POINTER(Options), ctypes.POINTER(vp)]
    lib.donof_ri_init_ex.restype = i
    lib.donof_ri_metric_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.donof_ri_metric_info.restype = i
    lib.donof_ri_transform.argtypes = [vp, vp, i]
    lib.donof_ri_jk_mo.argtypes = [vp, vp, vp]
    lib.donof_ri_jk_ao_batch.argtypes = [vp, vp, vp]
    lib.donof_ri_energy_lagrangian.argtypes = [vp, vp, vp, vp]
    lib.donof_ri_fetch.argtypes = [vp, i, vp, ctypes.c_size_t]
    lib.donof_ri_sync.argtypes = [vp]
    lib.donof_ri_destroy.argtypes = [vp]
    lib.donof_ri_strerror.argtypes = [i]
    lib.donof_ri_strerror.restype = ctypes.c_char_p
    lib.donof_ri_launch_count.argtypes = [vp]
    lib.donof_ri_launch_count.restype = ctypes.c_longlong
    lib.donof_ri_check_wait_timeout.argtypes = [vp, ctypes.c_longlong]
    lib.donof_ri_check_wait_timeout.restype = i
    lib.donof_ri_rhf.argtypes = [vp, i, d, vp, vp, vp, vp, vp]
    lib.donof_ri_rhf.restype = i
    lib.donof_ri_apply_rotation.argtypes = [vp, vp, vp]
    lib.donof_ri_apply_rotation.restype = i
    lib.donof_ri_jmo_noalloc.argtypes = [vp, i, i, vp, vp]
    lib.donof_ri_jmo_noalloc.restype = i
    lib.donof_ri_iteration.argtypes = [vp, vp, vp, i, vp, vp, vp, vp, i]
    lib.donof_ri_iteration.restype = i
    lib.donof_ri_profile.argtypes = [vp, i]
    lib.donof_ri_profile.restype = i
    lib.donof_ri_profile_read.argtypes = [vp, i, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong)]
    lib.donof_ri_profile_read.restype = i
    lib.donof_ri_optimize_occupations.argtypes = [vp, vp, i, d, d, vp, vp, vp]
    lib.donof_ri_optimize_occupations.restype = i
    lib.donof_ri_autotune.argtypes = [vp, i, vp, vp]
    lib.donof_ri_autotune.restype = i
    lib.donof_ri_set_schedule.argtypes = [vp, i, i, i]
    lib.donof_ri_exact_jk.argtypes = [vp, vp, vp, vp]
    lib.donof_ri_exact_jk.restype = i
    lib.donof_ri_energy_lagrangian_contracted.argtypes = [vp, vp, vp, vp]
    lib.donof_ri_energy_lagrangian_contracted.restype = i
    lib.donof_ri_flambda_step.argtypes = [vp, vp, i, d, vp, ctypes.POINTER(d), ctypes.POINTER(i)]
    lib.donof_ri_flambda_step.restype = i
    lib.donof_ri_set_schedule.restype = i
    lib.donof_ri_rotate_orbitals.argtypes = [vp, d, vp, vp]
    lib.donof_ri_rotate_orbitals.restype = i
    lib.donof_ri_on_features.argtypes = [vp, vp]
    lib.donof_ri_on_features.restype = i
    lib.donof_ri_gamma_guess.argtypes = [vp, vp, d, vp]
    lib.donof_ri_gamma_guess.restype = i
    f = ctypes.c_float
    lib.donof_mlp_create.argtypes = [i, i, i, i, vp, ctypes.POINTER(vp)]
    lib.donof_mlp_param_count.argtypes = [vp]
    lib.donof_mlp_param_count.restype = ctypes.c_longlong
    lib.donof_mlp_set_params.argtypes = [vp, vp]
    lib.donof_mlp_get_params.argtypes = [vp, vp]
    lib.donof_mlp_set_normalization.argtypes = [vp, vp, vp]
    lib.donof_mlp_forward.argtypes = [vp, vp, i, vp]
    lib.donof_mlp_loss_grad.argtypes = [vp, vp, vp, i, vp, vp]
    lib.donof_mlp_train_step.argtypes = [vp, vp, vp, i, f, f, vp]
    lib.donof_mlp_destroy.argtypes = [vp]
    for name in ("donof_mlp_create", "donof_mlp_set_params", "donof_mlp_get_params", "donof_mlp_set_normalization",
                 "donof_mlp_forward", "donof_mlp_loss_grad", "donof_mlp_train_step", "donof_mlp_destroy"):
        getattr(lib, name).restype = i
    for name in ("donof_ri_init", "donof_ri_transform", "donof_ri_jk_mo", "donof_ri_jk_ao_batch",
                 "donof_ri_energy_lagrangian", "donof_ri_fetch", "donof_ri_sync", "donof_ri_destroy"):
        getattr(lib, name).restype = i
    _lib = lib
    return lib


def strerror(status: int) -> str:
    return load().donof_ri_strerror(int(status)).decode()


def _ptr(x, dtype=np.float64):
    """Raw pointer of a numpy array, a torch tensor or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch
        want = torch.float64 if dtype == np.float64 else torch.int32
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)!r}")


def _check(rc: int, where: str):
    if rc != DONOF_RI_OK:
        raise DonofError(rc, where)


def donof_ri_init(system, subspace, weak_rank, precision: int = DONOF_RI_FP64, stream=None, metric=None,
                  metric_tol: float = 0.0):
    """Build a context for a system (attributes as in synthetic.System). Returns the handle.
    metric: None (plain Cholesky, donof_ri_init) or DONOF_RI_METRIC_* (donof_ri_init_ex)."""
    lib = load()
    keep = dict(
        xyz=np.ascontiguousarray(system.atom_xyz, dtype=np.float64),
        z=np.ascontiguousarray(system.atom_charge, dtype=np.float64),
        bfa=np.ascontiguousarray(system.bf_atom, dtype=np.int32),
        bfx=np.ascontiguousarray(system.bf_alpha, dtype=np.float64),
        axa=np.ascontiguousarray(system.aux_atom, dtype=np.int32),
        axx=np.ascontiguousarray(system.aux_alpha, dtype=np.float64),
        sub=np.ascontiguousarray(subspace, dtype=np.int32),
        rank=np.ascontiguousarray(weak_rank, dtype=np.int32),
    )
    s = System(int(system.bf_alpha.shape[0]), int(system.aux_alpha.shape[0]), int(system.atom_xyz.shape[0]),
               int(system.n_strong), int(system.n_weak_per),
               keep["xyz"].ctypes.data, keep["z"].ctypes.data, keep["bfa"].ctypes.data, keep["bfx"].ctypes.data,
               keep["axa"].ctypes.data, keep["axx"].ctypes.data, keep["sub"].ctypes.data, keep["rank"].ctypes.data)
    ctx = ctypes.c_void_p()
    st = None if stream is None else ctypes.c_void_p(int(stream))
    if metric is None:
        _check(lib.donof_ri_init(ctypes.byref(s), int(precision), st, ctypes.byref(ctx)), "donof_ri_init")
    else:
        opt = Options(int(metric), float(metric_tol))
        _check(lib.donof_ri_init_ex(ctypes.byref(s), int(precision), st, ctypes.byref(opt), ctypes.byref(ctx)),
               "donof_ri_init_ex")
    return ctx


def donof_ri_metric_info(ctx):
    """(2x2 pivot blocks, raised eigenvalues, interchanges) of the context's metric factorisation."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().donof_ri_metric_info(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "donof_ri_metric_info")
    return a.value, b.value, c.value


def donof_ri_transform(ctx, C, mode: int):
    _check(load().donof_ri_transform(ctx, _ptr(C), int(mode)), "donof_ri_transform")


def donof_ri_jk_mo(ctx, J=None, K=None):
    _check(load().donof_ri_jk_mo(ctx, _ptr(J), _ptr(K)), "donof_ri_jk_mo")


def donof_ri_jk_ao_batch(ctx, Jao=None, Kao=None):
    _check(load().donof_ri_jk_ao_batch(ctx, _ptr(Jao), _ptr(Kao)), "donof_ri_jk_ao_batch")


def donof_ri_energy_lagrangian(ctx, gamma, E=None, lam=None):
    _check(load().donof_ri_energy_lagrangian(ctx, _ptr(gamma), _ptr(E), _ptr(lam)),
           "donof_ri_energy_lagrangian")


def donof_ri_fetch(ctx, what: int, dst: np.ndarray):
    _check(load().donof_ri_fetch(ctx, int(what), _ptr(dst), dst.size), "donof_ri_fetch")


def donof_ri_sync(ctx):
    _check(load().donof_ri_sync(ctx), "donof_ri_sync")


def donof_ri_destroy(ctx):
    _check(load().donof_ri_destroy(ctx), "donof_ri_destroy")


def donof_ri_launch_count(ctx) -> int:
    return int(load().donof_ri_launch_count(ctx))


def donof_ri_check_wait_timeout(ctx, limit_ns: int):
    """Launch the bounded-wait check (reported as DONOF_RI_E_TIMEOUT by the next sync)."""
    _check(load().donof_ri_check_wait_timeout(ctx, int(limit_ns)), "donof_ri_check_wait_timeout")


def donof_ri_iteration(ctx, C, gamma, mode: int, J=None, K=None, E=None, lam=None, use_graph: bool = True):
    _check(load().donof_ri_iteration(ctx, _ptr(C), _ptr(gamma), int(mode), _ptr(J), _ptr(K), _ptr(E), _ptr(lam),
                                     1 if use_graph else 0), "donof_ri_iteration")


def donof_ri_jmo_noalloc(d, naux: int, n_omega: int, J, stream=None):
    """J from a device diagonal d [naux][n_omega] into device J, without device allocation."""
    st = None if stream is None else ctypes.c_void_p(int(stream))
    _check(load().donof_ri_jmo_noalloc(_ptr(d), int(naux), int(n_omega), _ptr(J), st), "donof_ri_jmo_noalloc")


def donof_ri_optimize_occupations(ctx, gamma, max_iter: int, gtol: float, etol: float = 0.0, E=None, grad=None,
                                  info=None):
    """Occupation optimisation for the current orbitals; gamma is updated in place."""
    ip = None if info is None else info.ctypes.data
    _check(load().donof_ri_optimize_occupations(ctx, _ptr(gamma), int(max_iter), float(gtol), float(etol), _ptr(E),
                                                _ptr(grad), ip), "donof_ri_optimize_occupations")


def donof_ri_rotate_orbitals_dev(ctx, radius: float, C_out, gmax_out: np.ndarray):
    """One rotation step; C_out a device tensor (column-major nbf*nbf) or None, gmax_out a 1-element float64 array."""
    _check(load().donof_ri_rotate_orbitals(ctx, float(radius), _ptr(C_out), gmax_out.ctypes.data),
           "donof_ri_rotate_orbitals")


def donof_ri_apply_rotation(ctx, kappa, C_out=None):
    """C <- C expm(kappa) (kappa row-major antisymmetric, numpy or device tensor); C_out optional."""
    _check(load().donof_ri_apply_rotation(ctx, _ptr(kappa), _ptr(C_out)), "donof_ri_apply_rotation")


def donof_ri_autotune(ctx, reps: int = 5):
    """Tune the SLICE4 tile schedule; returns (report [6, 4] int array, settings tried)."""
    rep = np.zeros(24, dtype=np.int32)
    tried = np.zeros(1, dtype=np.int32)
    _check(load().donof_ri_autotune(ctx, int(reps), rep.ctypes.data, tried.ctypes.data), "donof_ri_autotune")
    return rep.reshape(6, 4), int(tried[0])


def donof_ri_energy_lagrangian_contracted(ctx, gamma, E=None, lam=None):
    """E and lambda without the per-orbital AO matrices (after a FULL transform; FP64 contexts)."""
    _check(load().donof_ri_energy_lagrangian_contracted(ctx, _ptr(gamma), _ptr(E), _ptr(lam)),
           "donof_ri_energy_lagrangian_contracted")


def donof_ri_flambda_step(ctx, diag, first: bool, bound: float, C=None):
    """One F^lambda step: diag (float64 [nbf], in unless first, out: eigenvalues); returns (gmax, sweeps)."""
    g = ctypes.c_double()
    sw = ctypes.c_int()
    _check(load().donof_ri_flambda_step(ctx, _ptr(diag), 1 if first else 0, float(bound), _ptr(C), ctypes.byref(g),
                                        ctypes.byref(sw)), "donof_ri_flambda_step")
    return g.value, sw.value


def donof_ri_exact_jk(ctx, C, J=None, K=None):
    """Exact four-centre J, K (and J^(q), K^(q) kept in the context) for orbitals C."""
    _check(load().donof_ri_exact_jk(ctx, _ptr(C), _ptr(J), _ptr(K)), "donof_ri_exact_jk")


def donof_ri_set_schedule(ctx, kind: int, stages: int, option: int):
    """Set one GEMM kind's pipeline depth and option (see include/donof_ri.h)."""
    _check(load().donof_ri_set_schedule(ctx, int(kind), int(stages), int(option)), "donof_ri_set_schedule")


def donof_ri_profile(ctx, enable: bool):
    _check(load().donof_ri_profile(ctx, 1 if enable else 0), "donof_ri_profile")


def donof_ri_profile_read(ctx, row: int):
    """(total_ms, count) of the timed launch groups of one hot-path row since the last read."""
    t = ctypes.c_double()
    c = ctypes.c_longlong()
    _check(load().donof_ri_profile_read(ctx, int(row), ctypes.byref(t), ctypes.byref(c)), "donof_ri_profile_read")
    return t.value, c.value


def _fptr(x):
    """Pointer of a C-contiguous float32 numpy array or a contiguous float32 torch tensor."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float32 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float32 array")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise TypeError("expected a contiguous float32 tensor")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)!r}")


class Mlp:
    """The learned warm-start network (donof_mlp_*): FP32 arrays in and out."""

    def __init__(self, n_in: int, n_hidden: int, n_out: int, max_batch: int, stream=None):
        out = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(int(stream))
        _check(load().donof_mlp_create(int(n_in), int(n_hidden), int(n_out), int(max_batch), st, ctypes.byref(out)),
               "donof_mlp_create")
        self.ptr = out
        self.n_in, self.n_hidden, self.n_out = n_in, n_hidden, n_out
        self.nparam = int(load().donof_mlp_param_count(self.ptr))

    def close(self):
        if self.ptr is not None:
            load().donof_mlp_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.nparam
        _check(load().donof_mlp_set_params(self.ptr, _fptr(p)), "donof_mlp_set_params")

    def get_params(self) -> np.ndarray:
        p = np.empty(self.nparam, dtype=np.float32)
        _check(load().donof_mlp_get_params(self.ptr, _fptr(p)), "donof_mlp_get_params")
        return p

    def set_normalization(self, mean, inv_std):
        mu = np.ascontiguousarray(mean, dtype=np.float32)
        sd = np.ascontiguousarray(inv_std, dtype=np.float32)
        _check(load().donof_mlp_set_normalization(self.ptr, _fptr(mu), _fptr(sd)), "donof_mlp_set_normalization")

    def forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.empty((X.shape[0], self.n_out), dtype=np.float32)
        _check(load().donof_mlp_forward(self.ptr, _fptr(X), X.shape[0], _fptr(Y)), "donof_mlp_forward")
        return Y

    def loss_grad(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        g = np.empty(self.nparam, dtype=np.float32)
        _check(load().donof_mlp_loss_grad(self.ptr, _fptr(X), _fptr(T), X.shape[0], _fptr(loss), _fptr(g)),
               "donof_mlp_loss_grad")
        return float(loss[0]), g

    def train_step(self, X, T, lr: float, weight_decay: float = 0.0, loss_out=None):
        """One Adam step; X, T numpy (host) or torch (device) float32 tensors."""
        Xp = _fptr(X if not isinstance(X, np.ndarray) else np.ascontiguousarray(X, dtype=np.float32))
        Tp = _fptr(T if not isinstance(T, np.ndarray) else np.ascontiguousarray(T, dtype=np.float32))
        B = int(X.shape[0])
        _check(load().donof_mlp_train_step(self.ptr, Xp, Tp, B, float(lr), float(weight_decay), _fptr(loss_out)),
               "donof_mlp_train_step")


class Engine:
    """Convenience wrapper owning one context (host numpy in, host numpy out)."""

    def __init__(self, system, precision: int = DONOF_RI_FP64, stream=None, metric=None, metric_tol: float = 0.0):
        from synthetic import pairing_columns
        self.system = system
        self.nbf = int(system.bf_alpha.shape[0])
        self.naux = int(system.aux_alpha.shape[0])
        self.n_omega = int(system.n_strong * (1 + system.n_weak_per))
        self.subspace, self.weak_rank = pairing_columns(system.n_strong, system.n_weak_per)
        self.precision = int(precision)
        self.ctx = donof_ri_init(system, self.subspace, self.weak_rank, precision, stream, metric, metric_tol)

    def close(self):
        if self.ctx is not None:
            donof_ri_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def colmajor(C: np.ndarray) -> np.ndarray:
        """numpy [mu, p] orbital matrix -> the ABI's column-major buffer."""
        return np.ascontiguousarray(np.asarray(C, dtype=np.float64).T)

    def transform(self, C: np.ndarray, mode: int = DONOF_RI_FULL):
        donof_ri_transform(self.ctx, self.colmajor(C), mode)

    def jk_mo(self):
        m = self.n_omega
        J = np.empty((m, m))
        K = np.empty((m, m))
        donof_ri_jk_mo(self.ctx, J, K)
        return J, K

    def jk_ao(self, want=True):
        if not want:
            donof_ri_jk_ao_batch(self.ctx)
            return None
        m, nb = self.n_omega, self.nbf
        Jao = np.empty((m, nb, nb))
        Kao = np.empty((m, nb, nb))
        donof_ri_jk_ao_batch(self.ctx, Jao, Kao)
        return Jao, Kao

    def energy_lagrangian(self, gamma: np.ndarray):
        E = np.zeros(1)
        lam_cm = np.empty(self.nbf * self.nbf)
        donof_ri_energy_lagrangian(self.ctx, np.ascontiguousarray(gamma, dtype=np.float64), E, lam_cm)
        return float(E[0]), lam_cm.reshape(self.nbf, self.nbf).T.copy()

    def energy_lagrangian_contracted(self, gamma: np.ndarray):
        """E and lambda with F^(p) C_p straight from the transforms (no J^(q), K^(q))."""
        E = np.zeros(1)
        lam_cm = np.empty(self.nbf * self.nbf)
        donof_ri_energy_lagrangian_contracted(self.ctx, np.ascontiguousarray(gamma, dtype=np.float64), E, lam_cm)
        return float(E[0]), lam_cm.reshape(self.nbf, self.nbf).T.copy()

    def fetch(self, what: int) -> np.ndarray:
        nb, nx, m = self.nbf, self.naux, self.n_omega
        shapes = {
            DONOF_RI_FETCH_B: (nx, nb, nb), DONOF_RI_FETCH_BHALF: (nx, m, nb), DONOF_RI_FETCH_DIAG: (nx, m),
            DONOF_RI_FETCH_HCORE: (nb, nb), DONOF_RI_FETCH_OVERLAP: (nb, nb), DONOF_RI_FETCH_METRIC: (nx, nx),
            DONOF_RI_FETCH_ENUC: (1,), DONOF_RI_FETCH_OCC: (m,),
        }
        out = np.empty(shapes[what])
        donof_ri_fetch(self.ctx, what, out)
        return out

    def launches(self) -> int:
        return donof_ri_launch_count(self.ctx)

    def rhf(self, max_iter: int = 100, tol: float = 1e-9):
        """Closed-shell RI-HF orbitals (donof_ri_rhf): (C [mu, p], eps, E, iterations, commutator)."""
        nb = self.nbf
        Ccm = np.empty(nb * nb)
        eps = np.empty(nb)
        E = ctypes.c_double()
        it = ctypes.c_int()
        com = ctypes.c_double()
        _check(load().donof_ri_rhf(self.ctx, int(max_iter), float(tol), _ptr(Ccm), _ptr(eps), ctypes.byref(E),
                                   ctypes.byref(it), ctypes.byref(com)), "donof_ri_rhf")
        return Ccm.reshape(nb, nb).T.copy(), eps, E.value, it.value, com.value

    def overlap(self) -> np.ndarray:
        """The basis overlap matrix S the context evaluated at init."""
        return self.fetch(DONOF_RI_FETCH_OVERLAP)


    def optimize_occupations(self, gamma0: np.ndarray, max_iter: int = 5000, gtol: float = 1e-8,
                             etol: float = 1e-14):
        """(gamma, E, grad, iterations, stop reason) from the device L-BFGS (max_iter 0: evaluate only)."""
        g = np.array(gamma0, dtype=np.float64, copy=True)
        E = np.zeros(1)
        grad = np.empty_like(g)
        info = np.zeros(2, dtype=np.int32)
        donof_ri_optimize_occupations(self.ctx, g, max_iter, gtol, etol, E, grad, info)
        return g, float(E[0]), grad, int(info[0]), int(info[1])

    def rotate(self, radius: float):
        """One rotation step from the last energy_lagrangian: (rotated C [mu, p], max|lambda - lambda^T|)."""
        Ccm = np.empty(self.nbf * self.nbf)
        g = ctypes.c_double()
        _check(load().donof_ri_rotate_orbitals(self.ctx, float(radius), _ptr(Ccm), ctypes.byref(g)),
               "donof_ri_rotate_orbitals")
        return Ccm.reshape(self.nbf, self.nbf).T.copy(), g.value

    def on_features(self) -> np.ndarray:
        X = np.empty((self.system.n_strong, 3 + 4 * self.system.n_weak_per), dtype=np.float32)
        _check(load().donof_ri_on_features(self.ctx, _fptr(X)), "donof_ri_on_features")
        return X

    def gamma_guess(self, net: "Mlp", clip: float = 0.05) -> np.ndarray:
        g = np.empty(self.system.n_strong * self.system.n_weak_per)
        _check(load().donof_ri_gamma_guess(self.ctx, net.ptr, float(clip), _ptr(g)), "donof_ri_gamma_guess")
        return g


def engine_and_workload(name: str, precision: int = DONOF_RI_FP64, seed=None, stream=None):
    """A context for a named synthetic workload and the workload, whose orbitals
    C = S^-1/2 Q are built from the overlap matrix this context evaluated."""
    from synthetic import make_workload, workload_system
    eng = Engine(workload_system(name, seed), precision, stream=stream)
    return eng, make_workload(name, eng.overlap(), seed=seed)
