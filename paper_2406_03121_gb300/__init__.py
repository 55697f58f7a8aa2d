"""Python binding of ``libmess.so`` (include/mess.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays / torch tensors to
pointers and status codes to exceptions.  There is no CPU fallback: importing the package fails
loudly when the compiled library is missing (build it with ``paper_2406_03121_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmess.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libmess.so not built ({LIB_PATH}); run paper_2406_03121_gb300.build.build()")

_lib = ctypes.CDLL(LIB_PATH)

MESS_OK, MESS_EINVAL, MESS_ENOMEM, MESS_ECUDA = 0, -1, -2, -3
MESS_ENOCONV, MESS_ENUMERIC, MESS_ETIMEOUT, MESS_ENOTIMPL = -4, -5, -6, -7
MESS_FP64, MESS_MIXED, MESS_FP32 = 0, 1, 2
MESS_GUESS_CORE, MESS_GUESS_SAD, MESS_GUESS_MLP = 0, 1, 2
PRECISION = {"fp64": MESS_FP64, "mixed": MESS_MIXED, "fp32": MESS_FP32}

EXPORTED = [
    "mess_basis_create", "mess_basis_nbf", "mess_basis_nshell", "mess_basis_nelectron",
    "mess_basis_destroy", "mess_overlap", "mess_kinetic", "mess_nuclear", "mess_one_e_device",
    "mess_nuclear_repulsion", "mess_jk_build", "mess_jk_build_device", "mess_jk_build_static", "mess_eri_tensor",
    "mess_schwarz", "mess_scf", "mess_scf_batch", "mess_minimise", "mess_minimise_batch", "mess_xc", "mess_gradient", "mess_gradient_numerical", "mess_jk_profile", "mess_jk_autotune", "mess_jk_set_variant",
    "mess_jk_get_tuning", "mess_jk_set_tuning", "mess_boys_grid", "mess_profiler_range", "mess_fma_peak",
    "mess_last_error",
    "mess_mlp_num_params", "mess_mlp_create", "mess_mlp_destroy", "mess_mlp_get_params", "mess_mlp_set_params",
    "mess_mlp_save", "mess_mlp_load", "mess_mlp_features", "mess_mlp_loss_grad", "mess_mlp_train",
    "mess_mlp_predict",
]
MLP_DIN, MLP_WIDTH, MLP_DOUT = 112, 256, 25


class mess_jk_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("schwarz_tau", ctypes.c_double), ("fp64_tau", ctypes.c_double),
                ("boys_fp64", ctypes.c_int), ("split_df32", ctypes.c_int), ("cuda_stream", ctypes.c_void_p)]


class mess_jk_info(ctypes.Structure):
    _fields_ = [("shell_quartets", ctypes.c_longlong), ("function_quartets", ctypes.c_longlong),
                ("shell_quartets_fp64", ctypes.c_longlong), ("primitive_quartets", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class mess_jk_part(ctypes.Structure):
    _fields_ = [("qclass", ctypes.c_int), ("la", ctypes.c_int), ("lb", ctypes.c_int), ("lc", ctypes.c_int),
                ("ld", ctypes.c_int), ("fp64", ctypes.c_int), ("shell_quartets", ctypes.c_longlong),
                ("primitive_quartets", ctypes.c_longlong), ("function_quartets", ctypes.c_longlong),
                ("flops", ctypes.c_double), ("ms", ctypes.c_double), ("G", ctypes.c_int), ("team", ctypes.c_int),
                ("mode", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class mess_scf_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("guess", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("conv_E", ctypes.c_double), ("conv_comm", ctypes.c_double), ("diis_n", ctypes.c_int),
                ("schwarz_tau", ctypes.c_double), ("fp64_tau", ctypes.c_double), ("boys_fp64", ctypes.c_int),
                ("split_df32", ctypes.c_int), ("mlp_weights", ctypes.c_char_p), ("cuda_stream", ctypes.c_void_p),
                ("dens_tau", ctypes.c_double), ("xc", ctypes.c_int)]


class mess_min_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("steps", ctypes.c_int), ("lr", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("eps", ctypes.c_double), ("grad_tol", ctypes.c_double),
                ("schwarz_tau", ctypes.c_double), ("fp64_tau", ctypes.c_double), ("boys_fp64", ctypes.c_int),
                ("split_df32", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("xc", ctypes.c_int)]


class mess_scf_result(ctypes.Structure):
    _fields_ = [("E_total", ctypes.c_double), ("E_elec", ctypes.c_double), ("E_nuc", ctypes.c_double),
                ("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("E_iter", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


mess_basis_create = _sig("mess_basis_create", ctypes.c_int,
                         [ctypes.c_int, _IP, _DP, ctypes.c_char_p, ctypes.POINTER(_P)])
mess_basis_nbf = _sig("mess_basis_nbf", ctypes.c_int, [_P])
mess_basis_nshell = _sig("mess_basis_nshell", ctypes.c_int, [_P])
mess_basis_nelectron = _sig("mess_basis_nelectron", ctypes.c_int, [_P])
mess_basis_destroy = _sig("mess_basis_destroy", None, [_P])
mess_overlap = _sig("mess_overlap", ctypes.c_int, [_P, _DP])
mess_kinetic = _sig("mess_kinetic", ctypes.c_int, [_P, _DP])
mess_nuclear = _sig("mess_nuclear", ctypes.c_int, [_P, _DP])
mess_one_e_device = _sig("mess_one_e_device", ctypes.c_int, [_P, _P, _P, _P, _P])
mess_nuclear_repulsion = _sig("mess_nuclear_repulsion", ctypes.c_double, [_P])
mess_jk_build = _sig("mess_jk_build", ctypes.c_int,
                     [_P, _DP, _DP, _DP, ctypes.POINTER(mess_jk_opts), ctypes.POINTER(mess_jk_info)])
mess_jk_build_device = _sig("mess_jk_build_device", ctypes.c_int,
                            [_P, _P, _P, _P, ctypes.POINTER(mess_jk_opts), ctypes.POINTER(mess_jk_info)])
mess_jk_build_static = _sig("mess_jk_build_static", ctypes.c_int,
                            [_P, _DP, _DP, _DP, ctypes.POINTER(mess_jk_opts), ctypes.POINTER(mess_jk_info)])
mess_eri_tensor = _sig("mess_eri_tensor", ctypes.c_int, [_P, _DP])
mess_schwarz = _sig("mess_schwarz", ctypes.c_int, [_P, _DP])
mess_scf = _sig("mess_scf", ctypes.c_int,
                [_P, ctypes.POINTER(mess_scf_opts), ctypes.POINTER(mess_scf_result), _DP])
mess_scf_batch = _sig("mess_scf_batch", ctypes.c_int,
                      [ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(mess_scf_opts),
                       ctypes.POINTER(mess_scf_result)])
mess_minimise = _sig("mess_minimise", ctypes.c_int,
                     [_P, ctypes.POINTER(mess_min_opts), ctypes.POINTER(mess_scf_result), _DP])
mess_minimise_batch = _sig("mess_minimise_batch", ctypes.c_int,
                           [ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(mess_min_opts),
                            ctypes.POINTER(mess_scf_result), _DP])
mess_gradient = _sig("mess_gradient", ctypes.c_int,
                     [_P, ctypes.POINTER(mess_scf_opts), ctypes.POINTER(mess_scf_result), _DP])
mess_gradient_numerical = _sig("mess_gradient_numerical", ctypes.c_int,
                               [_P, ctypes.POINTER(mess_scf_opts), ctypes.POINTER(mess_scf_result), _DP])
mess_xc = _sig("mess_xc", ctypes.c_int, [_P, ctypes.c_int, _DP, _DP, _DP, ctypes.POINTER(ctypes.c_longlong)])
mess_jk_profile = _sig("mess_jk_profile", ctypes.c_int,
                       [_P, _P, _P, _P, ctypes.POINTER(mess_jk_opts), ctypes.POINTER(mess_jk_part), ctypes.c_int,
                        ctypes.POINTER(ctypes.c_int)])
mess_jk_autotune = _sig("mess_jk_autotune", ctypes.c_int,
                        [_P, _DP, ctypes.POINTER(mess_jk_opts), ctypes.c_int, ctypes.POINTER(ctypes.c_int)])
mess_jk_set_variant = _sig("mess_jk_set_variant", ctypes.c_int,
                           [_P, ctypes.POINTER(mess_jk_opts), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.POINTER(ctypes.c_int)])
mess_jk_get_tuning = _sig("mess_jk_get_tuning", ctypes.c_int,
                          [_P, ctypes.POINTER(mess_jk_opts), _IP, ctypes.c_int, _IP])
mess_jk_set_tuning = _sig("mess_jk_set_tuning", ctypes.c_int, [_P, ctypes.POINTER(mess_jk_opts), _IP, ctypes.c_int])
mess_boys_grid = _sig("mess_boys_grid", ctypes.c_int, [_DP, ctypes.c_int, _IP, _IP, _DP])
mess_profiler_range = _sig("mess_profiler_range", ctypes.c_int, [ctypes.c_int])
mess_fma_peak = _sig("mess_fma_peak", ctypes.c_int, [_DP, _DP, _P])
mess_last_error = _sig("mess_last_error", ctypes.c_char_p, [])
_FP = ctypes.POINTER(ctypes.c_float)
mess_mlp_num_params = _sig("mess_mlp_num_params", ctypes.c_int, [])
mess_mlp_create = _sig("mess_mlp_create", ctypes.c_int, [ctypes.c_ulonglong, ctypes.POINTER(_P)])
mess_mlp_destroy = _sig("mess_mlp_destroy", None, [_P])
mess_mlp_get_params = _sig("mess_mlp_get_params", ctypes.c_int, [_P, _FP])
mess_mlp_set_params = _sig("mess_mlp_set_params", ctypes.c_int, [_P, _FP])
mess_mlp_save = _sig("mess_mlp_save", ctypes.c_int, [_P, ctypes.c_char_p])
mess_mlp_load = _sig("mess_mlp_load", ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_P)])
mess_mlp_features = _sig("mess_mlp_features", ctypes.c_int,
                         [_P, _DP, _FP, _FP, _FP, ctypes.POINTER(ctypes.c_longlong)])
mess_mlp_loss_grad = _sig("mess_mlp_loss_grad", ctypes.c_int,
                          [_P, ctypes.c_longlong, _FP, _FP, _FP, _DP, _FP])
mess_mlp_train = _sig("mess_mlp_train", ctypes.c_int,
                      [_P, ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(mess_scf_opts), ctypes.c_int, ctypes.c_int,
                       ctypes.c_double, _DP])
mess_mlp_predict = _sig("mess_mlp_predict", ctypes.c_int, [_P, _P, _DP])


class MessError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = mess_last_error().decode(errors="replace")
        super().__init__(f"{where}: status {status}: {msg}")


def _check(st, where):
    if st != MESS_OK:
        raise MessError(st, where)


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _tptr(t):
    """device pointer of a contiguous float64 CUDA tensor"""
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def jk_opts(prec="fp64", schwarz_tau=0.0, fp64_tau=0.0, stream=None, boys_fp64=False, split_df32=False) -> mess_jk_opts:
    p = PRECISION[prec] if isinstance(prec, str) else int(prec)
    return mess_jk_opts(p, float(schwarz_tau), float(fp64_tau), int(bool(boys_fp64)), int(bool(split_df32)),
                        _stream_handle(stream))


class Basis:
    """A contracted Cartesian Gaussian basis of one structure (owns a ``mess_basis``)."""

    def __init__(self, Z, xyz_bohr, basis_file: str):
        Z = np.ascontiguousarray(np.asarray(Z, dtype=np.int32).ravel())
        xyz = np.ascontiguousarray(np.asarray(xyz_bohr, dtype=np.float64).reshape(-1, 3))
        if xyz.shape[0] != Z.shape[0]:
            raise ValueError("Z and xyz disagree on the atom count")
        h = _P()
        _check(mess_basis_create(int(Z.shape[0]), Z.ctypes.data_as(_IP), _dptr(xyz),
                                 os.fsencode(basis_file), ctypes.byref(h)), "mess_basis_create")
        self._h = h
        self.Z, self.xyz, self.basis_file = Z, xyz, basis_file

    @classmethod
    def from_molecule(cls, mol, basis_file: str):
        return cls(mol.Z, mol.xyz, basis_file)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            mess_basis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nbf(self) -> int:
        return int(mess_basis_nbf(self._h))

    @property
    def nshell(self) -> int:
        return int(mess_basis_nshell(self._h))

    @property
    def nelectron(self) -> int:
        return int(mess_basis_nelectron(self._h))

    def _mat(self, fn, name):
        out = np.zeros((self.nbf, self.nbf))
        _check(fn(self._h, _dptr(out)), name)
        return out

    def overlap(self):
        return self._mat(mess_overlap, "mess_overlap")

    def kinetic(self):
        return self._mat(mess_kinetic, "mess_kinetic")

    def nuclear(self):
        return self._mat(mess_nuclear, "mess_nuclear")

    def one_e_device(self, S=None, T=None, V=None, stream=None):
        ptr = lambda t: None if t is None else _tptr(t)  # noqa: E731
        _check(mess_one_e_device(self._h, ptr(S), ptr(T), ptr(V), _stream_handle(stream)), "mess_one_e_device")

    def nuclear_repulsion(self) -> float:
        return float(mess_nuclear_repulsion(self._h))

    def schwarz(self):
        out = np.zeros((self.nshell, self.nshell))
        _check(mess_schwarz(self._h, _dptr(out)), "mess_schwarz")
        return out

    def eri_tensor(self):
        n = self.nbf
        out = np.zeros((n, n, n, n))
        _check(mess_eri_tensor(self._h, _dptr(out)), "mess_eri_tensor")
        return out

    def jk(self, D, prec="fp64", schwarz_tau=0.0, fp64_tau=0.0, boys_fp64=False, split_df32=False, J=None, K=None):
        """J, K of a host density (numpy); returns (J, K, info dict).  J, K (optional): caller-owned
        C-contiguous float64 n x n outputs, e.g. views of page-locked host memory."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        for X in (J, K):
            if X is not None and (X.dtype != np.float64 or X.shape != D.shape or not X.flags.c_contiguous):
                raise ValueError("J and K must be C-contiguous float64 arrays shaped like D")
        J = np.zeros_like(D) if J is None else J
        K = np.zeros_like(D) if K is None else K
        info = mess_jk_info()
        o = jk_opts(prec, schwarz_tau, fp64_tau, None, boys_fp64, split_df32)
        _check(mess_jk_build(self._h, _dptr(D), _dptr(J), _dptr(K), ctypes.byref(o), ctypes.byref(info)),
               "mess_jk_build")
        return J, K, info.as_dict()

    def jk_autotune(self, D, prec="fp64", schwarz_tau=0.0, fp64_tau=0.0, boys_fp64=False, split_df32=False, reps=3,
                    stream=None):
        """Time every kernel variant of each bin part on host density D and keep the fastest for later
        builds with these options; returns the number of parts whose kernel changed."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        o = jk_opts(prec, schwarz_tau, fp64_tau, stream, boys_fp64, split_df32)
        n = ctypes.c_int()
        _check(mess_jk_autotune(self._h, _dptr(D), ctypes.byref(o), int(reps), ctypes.byref(n)), "mess_jk_autotune")
        return n.value

    def jk_set_variant(self, G=1, team=0, split_mode=-1, prec="fp64", schwarz_tau=0.0, fp64_tau=0.0,
                       boys_fp64=False, split_df32=False):
        """Force one kernel variant on every bin part of these options (see mess_jk_set_variant)."""
        o = jk_opts(prec, schwarz_tau, fp64_tau, None, boys_fp64, split_df32)
        n = ctypes.c_int()
        _check(mess_jk_set_variant(self._h, ctypes.byref(o), int(G), int(team), int(split_mode),
                                   ctypes.byref(n)), "mess_jk_set_variant")
        return n.value

    def jk_tuning(self, prec="fp64", schwarz_tau=0.0, fp64_tau=0.0, boys_fp64=False, split_df32=False):
        """Kernel choice per bin part: a list of [class, G, team, arithmetic]."""
        o = jk_opts(prec, schwarz_tau, fp64_tau, None, boys_fp64, split_df32)
        n = ctypes.c_int()
        _check(mess_jk_get_tuning(self._h, ctypes.byref(o), None, 0, ctypes.byref(n)), "mess_jk_get_tuning")
        t = np.zeros(4 * n.value, dtype=np.int32)
        _check(mess_jk_get_tuning(self._h, ctypes.byref(o), t.ctypes.data_as(_IP), n.value, ctypes.byref(n)),
               "mess_jk_get_tuning")
        return t.reshape(-1, 4).tolist()

    def jk_set_tuning(self, table, prec="fp64", schwarz_tau=0.0, fp64_tau=0.0, boys_fp64=False, split_df32=False):
        """Restore a kernel choice saved by jk_tuning (same basis and options)."""
        o = jk_opts(prec, schwarz_tau, fp64_tau, None, boys_fp64, split_df32)
        t = np.ascontiguousarray(np.asarray(table, dtype=np.int32).reshape(-1))
        _check(mess_jk_set_tuning(self._h, ctypes.byref(o), t.ctypes.data_as(_IP), len(t) // 4), "mess_jk_set_tuning")

    def jk_device(self, D, J, K, prec="fp64", schwarz_tau=0.0, fp64_tau=0.0, stream=None, boys_fp64=False,
                  split_df32=False):
        """J, K of a device density (torch float64 CUDA tensors, caller-owned); enqueued on stream."""
        info = mess_jk_info()
        o = jk_opts(prec, schwarz_tau, fp64_tau, stream, boys_fp64, split_df32)
        _check(mess_jk_build_device(self._h, _tptr(D), _tptr(J), _tptr(K), ctypes.byref(o), ctypes.byref(info)),
               "mess_jk_build_device")
        return info.as_dict()

    def jk_profile(self, D, J, K, prec="fp64", schwarz_tau=0.0, fp64_tau=0.0, stream=None, boys_fp64=False,
                   split_df32=False):
        """Per-launch timings (CUDA events) and algorithmic flops of one device J/K build."""
        parts = (mess_jk_part * 1024)()
        n = ctypes.c_int()
        o = jk_opts(prec, schwarz_tau, fp64_tau, stream, boys_fp64, split_df32)
        _check(mess_jk_profile(self._h, _tptr(D), _tptr(J), _tptr(K), ctypes.byref(o), parts, 1024, ctypes.byref(n)),
               "mess_jk_profile")
        return [parts[i].as_dict() for i in range(n.value)]

    def gradient(self, numerical=False, **scf_kw):
        """SCF energy and nuclear gradient (natom x 3, hartree/bohr): mess_gradient (analytic where it
        applies), or mess_gradient_numerical with numerical=True."""
        o = scf_opts(**scf_kw)
        r = mess_scf_result()
        g = np.zeros((len(self.Z), 3))
        fn, name = (mess_gradient_numerical, "mess_gradient_numerical") if numerical else (mess_gradient, "mess_gradient")
        _check(fn(self._h, ctypes.byref(o), ctypes.byref(r), _dptr(g)), name)
        return r.as_dict(), g

    def xc(self, D, kind="lda"):
        """E_xc and V_xc of a host density on the library's grid (see mess_xc); returns (E_xc, V, points)."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        V = np.zeros_like(D)
        E = np.zeros(1)
        npts = ctypes.c_longlong()
        _check(mess_xc(self._h, XC[kind] if isinstance(kind, str) else int(kind), _dptr(D), _dptr(E), _dptr(V),
                       ctypes.byref(npts)), "mess_xc")
        return float(E[0]), V, npts.value

    def minimise(self, **kw):
        """Direct minimisation of this molecule's energy (see mess_minimise); returns (result dict,
        energy per step, status)."""
        o = min_opts(**kw)
        r = mess_scf_result()
        trace = np.zeros(o.steps)
        st = mess_minimise(self._h, ctypes.byref(o), ctypes.byref(r), _dptr(trace))
        if st not in (MESS_OK, MESS_ENOCONV):
            _check(st, "mess_minimise")
        return r.as_dict(), trace, st

    def scf(self, prec="fp64", guess=MESS_GUESS_CORE, max_iter=100, conv_E=1e-10, conv_comm=1e-8, diis_n=8,
            schwarz_tau=0.0, fp64_tau=0.0, mlp_weights=None, stream=None, want_density=True, boys_fp64=False,
            split_df32=False, dens_tau=0.0, xc="hf"):
        o = scf_opts(prec, guess, max_iter, conv_E, conv_comm, diis_n, schwarz_tau, fp64_tau, mlp_weights, stream,
                     boys_fp64, split_df32, dens_tau, xc)
        res = mess_scf_result()
        D = np.zeros((self.nbf, self.nbf)) if want_density else None
        st = mess_scf(self._h, ctypes.byref(o), ctypes.byref(res), _dptr(D) if D is not None else None)
        if st not in (MESS_OK, MESS_ENOCONV):
            _check(st, "mess_scf")
        out = res.as_dict()
        out["status"] = st
        out["D"] = D
        return out


def boys_grid():
    """The kernels' Boys-function grid: (table [rows, 17] = F_0..F_15 and exp(-T) per row, dT)."""
    nr, nc, dT = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(mess_boys_grid(None, 0, ctypes.byref(nr), ctypes.byref(nc), ctypes.byref(dT)), "mess_boys_grid")
    t = np.zeros((nr.value, nc.value))
    _check(mess_boys_grid(_dptr(t), t.size, None, None, None), "mess_boys_grid")
    return t, dT.value


def profiler_range(on):
    """Start (True) or stop (False) the region recorded by a profiler launched with profiling off."""
    _check(mess_profiler_range(int(bool(on))), "mess_profiler_range")


def fma_peak(stream=None):
    """Measured FP32 and FP64 CUDA-core FMA throughput in TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(mess_fma_peak(ctypes.byref(a), ctypes.byref(b), _stream_handle(stream)), "mess_fma_peak")
    return a.value, b.value


XC = {"hf": 0, "hfx": 0, "lda": 1, "pbe": 2}


def scf_opts(prec="fp64", guess=MESS_GUESS_CORE, max_iter=100, conv_E=1e-10, conv_comm=1e-8, diis_n=8,
             schwarz_tau=0.0, fp64_tau=0.0, mlp_weights=None, stream=None, boys_fp64=False,
             split_df32=False, dens_tau=0.0, xc="hf") -> mess_scf_opts:
    p = PRECISION[prec] if isinstance(prec, str) else int(prec)
    w = os.fsencode(mlp_weights) if mlp_weights else None
    return mess_scf_opts(p, int(guess), int(max_iter), float(conv_E), float(conv_comm), int(diis_n),
                         float(schwarz_tau), float(fp64_tau), int(bool(boys_fp64)), int(bool(split_df32)), w,
                         _stream_handle(stream), float(dens_tau), XC[xc] if isinstance(xc, str) else int(xc))


def scf_batch(bases, prec="fp64", guess=MESS_GUESS_CORE, max_iter=100, conv_E=1e-10, conv_comm=1e-8,
              diis_n=8, schwarz_tau=0.0, fp64_tau=0.0, mlp_weights=None, stream=None, boys_fp64=False,
              split_df32=False, dens_tau=0.0, xc="hf"):
    """Batched SCF over many bases; returns a list of result dicts and the call's status."""
    n = len(bases)
    arr = (_P * n)(*[b.handle for b in bases])
    res = (mess_scf_result * n)()
    o = scf_opts(prec, guess, max_iter, conv_E, conv_comm, diis_n, schwarz_tau, fp64_tau, mlp_weights, stream,
                 boys_fp64, split_df32, dens_tau, xc)
    st = mess_scf_batch(n, arr, ctypes.byref(o), res)
    if st not in (MESS_OK, MESS_ENOCONV):
        _check(st, "mess_scf_batch")
    return [r.as_dict() for r in res], st


def min_opts(prec="fp64", steps=200, lr=0.1, beta1=0.9, beta2=0.999, eps=1e-8, grad_tol=1e-5, schwarz_tau=0.0,
             fp64_tau=0.0, boys_fp64=False, split_df32=False, stream=None, xc="hf") -> mess_min_opts:
    p = PRECISION[prec] if isinstance(prec, str) else int(prec)
    return mess_min_opts(p, int(steps), float(lr), float(beta1), float(beta2), float(eps), float(grad_tol),
                         float(schwarz_tau), float(fp64_tau), int(bool(boys_fp64)), int(bool(split_df32)),
                         _stream_handle(stream), XC[xc] if isinstance(xc, str) else int(xc))


def minimise_batch(bases, **kw):
    """Direct minimisation (QR-orthonormalised parameters, Adam) of every basis at once; returns (list
    of result dicts, energy trace as a steps x nmol array, status)."""
    n = len(bases)
    o = min_opts(**kw)
    arr = (_P * n)(*[b.handle for b in bases])
    res = (mess_scf_result * n)()
    trace = np.zeros((o.steps, n))
    st = mess_minimise_batch(n, arr, ctypes.byref(o), res, _dptr(trace))
    if st not in (MESS_OK, MESS_ENOCONV):
        _check(st, "mess_minimise_batch")
    return [r.as_dict() for r in res], trace, st


def _fptr(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(_FP)


class MLP:
    """The learned-guess network (owns a ``mess_mlp``)."""

    def __init__(self, seed: int = 1, path: str | None = None):
        h = _P()
        if path is None:
            _check(mess_mlp_create(ctypes.c_ulonglong(seed), ctypes.byref(h)), "mess_mlp_create")
        else:
            _check(mess_mlp_load(os.fsencode(path), ctypes.byref(h)), "mess_mlp_load")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            mess_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def num_params() -> int:
        return int(mess_mlp_num_params())

    def get_params(self):
        out = np.zeros(self.num_params(), dtype=np.float32)
        _check(mess_mlp_get_params(self._h, _fptr(out)), "mess_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(mess_mlp_set_params(self._h, _fptr(p)), "mess_mlp_set_params")

    def save(self, path):
        _check(mess_mlp_save(self._h, os.fsencode(path)), "mess_mlp_save")

    def loss_grad(self, X, T, M):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        M = np.ascontiguousarray(M, dtype=np.float32)
        loss = ctypes.c_double()
        g = np.zeros(self.num_params(), dtype=np.float32)
        _check(mess_mlp_loss_grad(self._h, X.shape[0], _fptr(X), _fptr(T), _fptr(M), ctypes.byref(loss), _fptr(g)),
               "mess_mlp_loss_grad")
        return loss.value, g

    def train(self, bases, epochs=10, batch_rows=8192, lr=1e-3, **scf_kw):
        n = len(bases)
        arr = (_P * n)(*[b.handle for b in bases])
        o = scf_opts(**scf_kw)
        losses = np.zeros(epochs)
        _check(mess_mlp_train(self._h, n, arr, ctypes.byref(o), epochs, batch_rows, lr, _dptr(losses)),
               "mess_mlp_train")
        return losses

    def predict(self, basis):
        D0 = np.zeros((basis.nbf, basis.nbf))
        _check(mess_mlp_predict(self._h, basis.handle, _dptr(D0)), "mess_mlp_predict")
        return D0


def mlp_features(basis, D=None):
    """(X, T, M) descriptors / pair-frame targets / masks of one molecule (T, M None without D)."""
    n = ctypes.c_longlong()
    _check(mess_mlp_features(basis.handle, None, None, None, None, ctypes.byref(n)), "mess_mlp_features")
    rows = n.value
    X = np.zeros((rows, MLP_DIN), dtype=np.float32)
    if D is None:
        _check(mess_mlp_features(basis.handle, None, _fptr(X), None, None, ctypes.byref(n)), "mess_mlp_features")
        return X, None, None
    D = np.ascontiguousarray(D, dtype=np.float64)
    T = np.zeros((rows, MLP_DOUT), dtype=np.float32)
    M = np.zeros((rows, MLP_DOUT), dtype=np.float32)
    _check(mess_mlp_features(basis.handle, _dptr(D), _fptr(X), _fptr(T), _fptr(M), ctypes.byref(n)),
           "mess_mlp_features")
    return X, T, M
