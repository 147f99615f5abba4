"""Python binding of the C ABI in include/fmo_xtb.h (argument marshalling only).

Every step of the FMO-xTB calculation runs in the CUDA library
``libfmo_xtb.so``; this module converts the parameter table, the system and
the options to the C structures, calls the library and returns NumPy arrays.
It fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from .inputs.params import MAX_PRIM, MAX_SHELL, MAX_Z, Params

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfmo_xtb.so")

FMO_OK = 0
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NOT_CONVERGED",
                5: "ERR_TIMEOUT", 6: "ERR_NAN", 7: "ERR_STATE", 8: "ERR_UNSUPPORTED", 9: "ERR_EXCHANGE"}
PREC_FP64, PREC_MIXED = 0, 1

SYMBOLS = ["fmo_options_default", "fmo_create", "fmo_set_system", "fmo_set_coordinates",
           "fmo_set_coordinates_device", "fmo_set_guess", "fmo_run", "fmo_get_energy",
           "fmo_get_sizes", "fmo_get_monomers", "fmo_get_dimers", "fmo_get_trimers", "fmo_get_gradient",
           "fmo_get_stats", "fmo_last_error", "fmo_destroy", "fmo_mlp_init", "fmo_mlp_set_weights",
           "fmo_mlp_get_weights", "fmo_mlp_predict", "fmo_mlp_train", "fmo_scc_solve_noalloc", "fmo_fma_peak",
           "fmo_mlp_loss_grad", "fmo_set_exchange", "fmo_lpt_partition", "fmo_sp2_projector",
           "fmo_sp2_projector_f32"]
MLP_N_WEIGHTS = 26908
MLP_N_TRAINED = 26754


class FmoElement(C.Structure):
    _fields_ = [("n_shell", C.c_int32), ("l", C.c_int32 * MAX_SHELL),
                ("n_prim", C.c_int32 * MAX_SHELL), ("pad_", C.c_int32),
                ("alpha", (C.c_double * MAX_PRIM) * MAX_SHELL),
                ("coef", (C.c_double * MAX_PRIM) * MAX_SHELL),
                ("h_l", C.c_double * MAX_SHELL), ("k_cn_l", C.c_double * MAX_SHELL),
                ("k_poly_l", C.c_double * MAX_SHELL), ("kappa_l", C.c_double * MAX_SHELL),
                ("q0_l", C.c_double * MAX_SHELL), ("eta", C.c_double), ("gamma3", C.c_double),
                ("en", C.c_double), ("r_cov", C.c_double), ("z_eff", C.c_double),
                ("alpha_rep", C.c_double)]


class FmoParams(C.Structure):
    _fields_ = [("el", FmoElement * MAX_Z), ("k_l", C.c_double * 3),
                ("k_ab", (C.c_double * MAX_Z) * MAX_Z), ("k_en", C.c_double),
                ("k_g", C.c_double), ("k_f", C.c_double), ("cn_k1", C.c_double),
                ("cn_k2", C.c_double), ("cn_cutoff", C.c_double), ("t_el", C.c_double),
                ("v_hop", C.c_double)]


class FmoOptions(C.Structure):
    _fields_ = [("level", C.c_int32), ("precision", C.c_int32), ("all_dimers_scc", C.c_int32),
                ("max_iter", C.c_int32), ("max_outer", C.c_int32), ("guess", C.c_int32),
                ("schedule", C.c_int32), ("monomer_loop", C.c_int32), ("dimer_cut", C.c_double),
                ("trimer_cut", C.c_double), ("scc_tol", C.c_double), ("e_tol", C.c_double),
                ("outer_tol", C.c_double), ("mixed_switch_tol", C.c_double),
                ("deadline_s", C.c_double), ("mixed_finish", C.c_int32), ("nmer_finish", C.c_int32),
                ("want_gradient", C.c_int32), ("esp_mode", C.c_int32), ("shard_rank", C.c_int32),
                ("shard_world", C.c_int32), ("nmer_ctas_per_sm", C.c_int32), ("nmer_matrix_smem", C.c_int32),
                ("monomer_ctas_per_sm", C.c_int32), ("monomer_matrix_smem", C.c_int32)]

# element-wise sum over the ranks of a sharded run (fmo_exchange_fn)
EXCHANGE_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.POINTER(C.c_double), C.c_int64)


class FmoStats(C.Structure):
    _fields_ = [("n_monomer_solves", C.c_int64), ("n_dimer_scc", C.c_int64),
                ("n_dimer_esdim", C.c_int64), ("n_trimer_scc", C.c_int64),
                ("scc_iterations", C.c_int64), ("kernel_launches", C.c_int64),
                ("outer_iterations", C.c_int32), ("n_failed", C.c_int32),
                ("ms_setup", C.c_double), ("ms_monomer", C.c_double), ("ms_select", C.c_double),
                ("ms_dimer", C.c_double), ("ms_trimer", C.c_double), ("ms_reduce", C.c_double),
                ("ms_scc", C.c_double * 3), ("scc_launches", C.c_int64 * 3),
                ("iters_fp32", C.c_int64 * 3), ("iters_fp64", C.c_int64 * 3),
                ("flops_fp32", C.c_double * 3), ("flops_fp64", C.c_double * 3),
                ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64), ("ms_gradient", C.c_double),
                ("zvector_iterations", C.c_int32), ("guess_restarts", C.c_int32),
                ("zvector_residual", C.c_double)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if hasattr(v, "__len__") else v
        return out


_lib_handle = None


def load_library(path: str | None = None):
    """Load libfmo_xtb.so (built by paper_2606_28022_b300.build)."""
    global _lib_handle
    if _lib_handle is not None and path is None:
        return _lib_handle
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} is missing "
                           "(run python -m paper_2606_28022_b300.build)")
    lib = C.CDLL(p)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    lib.fmo_options_default.argtypes = [C.POINTER(FmoOptions)]
    lib.fmo_options_default.restype = None
    lib.fmo_create.argtypes = [C.POINTER(vp), C.POINTER(FmoParams), C.c_int]
    lib.fmo_set_system.argtypes = [vp, i32, ip, dp, i32, ip, ip, i32, ip]
    lib.fmo_set_coordinates.argtypes = [vp, dp]
    lib.fmo_set_coordinates_device.argtypes = [vp, vp, vp]
    lib.fmo_set_guess.argtypes = [vp, dp]
    lib.fmo_run.argtypes = [vp, C.POINTER(FmoOptions), vp]
    lib.fmo_get_energy.argtypes = [vp, dp, dp, dp]
    lib.fmo_get_sizes.argtypes = [vp, ip, ip]
    lib.fmo_get_monomers.argtypes = [vp, dp, dp, ip, ip]
    lib.fmo_get_dimers.argtypes = [vp, C.POINTER(i64), ip, dp, dp, dp, C.POINTER(C.c_uint8), ip]
    lib.fmo_get_trimers.argtypes = [vp, C.POINTER(i64), ip, dp, dp]
    lib.fmo_get_gradient.argtypes = [vp, dp]
    lib.fmo_get_stats.argtypes = [vp, C.POINTER(FmoStats)]
    fp = C.POINTER(C.c_float)
    lib.fmo_mlp_init.argtypes = [vp, C.c_uint64]
    lib.fmo_mlp_set_weights.argtypes = [vp, fp, i64]
    lib.fmo_mlp_get_weights.argtypes = [vp, fp, C.POINTER(i64)]
    lib.fmo_mlp_predict.argtypes = [vp, dp]
    lib.fmo_mlp_train.argtypes = [vp, i32, dp, dp, i32, i32, C.c_double, C.c_uint64, dp]
    lib.fmo_mlp_loss_grad.argtypes = [vp, i32, dp, dp, dp, fp]
    lib.fmo_fma_peak.argtypes = [i32, i32, C.POINTER(C.c_double)]
    lib.fmo_set_exchange.argtypes = [vp, EXCHANGE_FN, vp]
    lib.fmo_lpt_partition.argtypes = [dp, i64, i32, ip]
    lib.fmo_scc_solve_noalloc.argtypes = [vp, i32, ip, vp, i32, vp, vp, vp, vp, vp, vp, C.c_char_p, i32]
    lib.fmo_sp2_projector.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, vp]
    lib.fmo_sp2_projector_f32.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, vp]
    lib.fmo_last_error.argtypes = [vp]
    lib.fmo_last_error.restype = C.c_char_p
    lib.fmo_destroy.argtypes = [vp]
    lib.fmo_destroy.restype = None
    for name in SYMBOLS:
        if name not in ("fmo_options_default", "fmo_last_error", "fmo_destroy"):
            getattr(lib, name).restype = C.c_int
    if path is None:
        _lib_handle = lib
    return lib


def fma_peak(precision: str = "fp32", device: int = 0) -> float:
    """Measured FMA throughput of the device in TFLOP/s (fmo_fma_peak)."""
    t = C.c_double(0.0)
    st = load_library().fmo_fma_peak(PREC_FP64 if precision == "fp64" else PREC_MIXED, device, C.byref(t))
    if st != FMO_OK:
        raise FMOError(st, "fmo_fma_peak failed")
    return t.value


def sp2_projector(F_ptr: int, n_occ_ptr: int, n: int, batch: int, max_iter: int, D_ptr: int,
                  work_ptr: int, iters_ptr: int, stream: int | None = None, fp32: bool = False) -> None:
    """Occupied-subspace projectors of a batch of symmetric n x n matrices by
    SP2 purification (fmo_sp2_projector, or fmo_sp2_projector_f32 on float
    buffers with fp32=True); every pointer is a device address."""
    lib = load_library()
    fn = lib.fmo_sp2_projector_f32 if fp32 else lib.fmo_sp2_projector
    st = fn(C.c_void_p(F_ptr), C.c_void_p(n_occ_ptr), int(n), int(batch), int(max_iter),
            C.c_void_p(D_ptr), C.c_void_p(work_ptr), C.c_void_p(iters_ptr), C.c_void_p(stream or 0))
    if st != FMO_OK:
        raise FMOError(st, "fmo_sp2_projector failed")


def lpt_partition(cost, world: int) -> np.ndarray:
    """Rank of every work unit under the library's LPT partition (fmo_lpt_partition)."""
    c = np.ascontiguousarray(cost, dtype=np.float64)
    owner = np.zeros(len(c), dtype=np.int32)
    st = load_library().fmo_lpt_partition(_dp(c), len(c), int(world), _ip(owner))
    if st != FMO_OK:
        raise FMOError(st, "fmo_lpt_partition failed")
    return owner


def params_to_c(params: Params) -> FmoParams:
    """Copy a parameter table into the C structure fmo_params."""
    cp = FmoParams()
    for z, el in params.elements.items():
        e = cp.el[z]
        e.n_shell = el.n_shell
        for k, l in enumerate(el.shells_l):
            e.l[k] = l
            a = np.asarray(el.alpha[k], dtype=np.float64)
            c = np.asarray(el.coef[k], dtype=np.float64)
            if len(a) > MAX_PRIM:
                raise ValueError("too many primitives in a shell")
            e.n_prim[k] = len(a)
            for p in range(len(a)):
                e.alpha[k][p] = a[p]
                e.coef[k][p] = c[p]
            e.h_l[k] = el.h_l[k]
            e.k_cn_l[k] = el.k_cn_l[k]
            e.k_poly_l[k] = el.k_poly_l[k]
            e.kappa_l[k] = el.kappa_l[k]
            e.q0_l[k] = el.q0_l[k]
        e.eta, e.gamma3, e.en = el.eta, el.gamma3, el.en
        e.r_cov, e.z_eff, e.alpha_rep = el.r_cov, el.z_eff, el.alpha_rep
    for l in range(3):
        cp.k_l[l] = params.k_l[l]
    kab = params.k_ab_matrix()
    for a in range(MAX_Z):
        row = cp.k_ab[a]
        for b in range(MAX_Z):
            row[b] = kab[a, b]
    cp.k_en, cp.k_g, cp.k_f = params.k_en, params.k_g, params.k_f
    cp.cn_k1, cp.cn_k2, cp.cn_cutoff = params.cn_k1, params.cn_k2, params.cn_cutoff
    cp.t_el, cp.v_hop = params.t_el, params.v_hop
    return cp


def options(**kw) -> FmoOptions:
    """fmo_options with the library defaults, overridden by keywords."""
    o = FmoOptions()
    load_library().fmo_options_default(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[v]
        if k == "monomer_loop" and isinstance(v, str):
            v = {"global": 0, "nested": 1}[v]
        if k == "nmer_finish" and isinstance(v, str):
            v = {"energy": 0, "iterate": 1}[v]
        if k == "esp_mode" and isinstance(v, str):
            v = {"auto": 0, "pairwise": 1}[v]
        setattr(o, k, v)
    return o


class FMOError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


@dataclasses.dataclass
class Monomers:
    energy: np.ndarray
    shell_dq: np.ndarray
    iters: np.ndarray
    status: np.ndarray


@dataclasses.dataclass
class Dimers:
    ij: np.ndarray
    dE: np.ndarray
    e_dimer: np.ndarray
    dEV: np.ndarray
    scc: np.ndarray
    iters: np.ndarray


@dataclasses.dataclass
class Trimers:
    ijk: np.ndarray
    dE3: np.ndarray
    corr: np.ndarray


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


class FMO:
    """One library context on one CUDA device."""

    def __init__(self, params: Params, device: int = 0):
        self.lib = load_library()
        self._cparams = params_to_c(params)
        h = C.c_void_p()
        st = self.lib.fmo_create(C.byref(h), C.byref(self._cparams), device)
        if st != FMO_OK:
            raise FMOError(st, "fmo_create failed")
        self.h = h
        self._exchange = None
        self.n_atoms = 0
        self.n_frag = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.fmo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=()):
        if st != FMO_OK and st not in allow:
            raise FMOError(st, self.lib.fmo_last_error(self.h).decode())
        return st

    def set_system(self, system):
        Z = np.ascontiguousarray(system.Z, dtype=np.int32)
        xyz = np.ascontiguousarray(system.xyz, dtype=np.float64).reshape(-1)
        frag = np.ascontiguousarray(system.frag, dtype=np.int32)
        chg = np.ascontiguousarray(system.frag_charge, dtype=np.int32)
        cut = np.ascontiguousarray(system.cut_bonds, dtype=np.int32).reshape(-1)
        self._check(self.lib.fmo_set_system(self.h, len(Z), _ip(Z), _dp(xyz), len(chg), _ip(frag),
                                            _ip(chg), len(cut) // 2, _ip(cut) if len(cut) else None))
        self.n_atoms, self.n_frag = len(Z), len(chg)

    def set_coordinates(self, xyz_host: np.ndarray):
        x = np.ascontiguousarray(xyz_host, dtype=np.float64).reshape(-1)
        self._check(self.lib.fmo_set_coordinates(self.h, _dp(x)))

    def set_coordinates_device(self, ptr: int, stream: int | None = None):
        self._check(self.lib.fmo_set_coordinates_device(self.h, C.c_void_p(ptr), C.c_void_p(stream or 0)))

    def set_exchange(self, fn):
        """Sharded runs: fn(buf) must replace the float64 array buf by its
        element-wise sum over all ranks (e.g. shard.allreduce_exchange)."""
        if fn is None:
            self._exchange = None
            self._check(self.lib.fmo_set_exchange(self.h, EXCHANGE_FN(), None))
            return

        def cb(user, ptr, n):
            try:
                fn(np.ctypeslib.as_array(ptr, shape=(int(n),)))
                return 0
            except Exception:   # noqa: BLE001 - reported to the library as a failed exchange
                return 1
        self._exchange = EXCHANGE_FN(cb)   # kept alive as long as the context
        self._check(self.lib.fmo_set_exchange(self.h, self._exchange, None))

    def set_guess(self, shell_dq: np.ndarray):
        x = np.ascontiguousarray(shell_dq, dtype=np.float64)
        self._check(self.lib.fmo_set_guess(self.h, _dp(x)))

    def run(self, opts: FmoOptions | None = None, stream: int | None = None, allow_unconverged=False):
        opts = options() if opts is None else opts
        allow = (4,) if allow_unconverged else ()
        return self._check(self.lib.fmo_run(self.h, C.byref(opts), C.c_void_p(stream or 0)), allow)

    def energies(self):
        e = np.zeros(3)
        self._check(self.lib.fmo_get_energy(self.h, _dp(e[0:]), _dp(e[1:]), _dp(e[2:])))
        return float(e[0]), float(e[1]), float(e[2])

    def sizes(self):
        ns, na = C.c_int32(), C.c_int32()
        self._check(self.lib.fmo_get_sizes(self.h, C.byref(ns), C.byref(na)))
        return ns.value, na.value

    def monomers(self) -> Monomers:
        ns, _ = self.sizes()
        E = np.zeros(self.n_frag)
        dq = np.zeros(ns)
        it = np.zeros(self.n_frag, dtype=np.int32)
        st = np.zeros(self.n_frag, dtype=np.int32)
        self._check(self.lib.fmo_get_monomers(self.h, _dp(E), _dp(dq), _ip(it), _ip(st)))
        return Monomers(E, dq, it, st)

    def dimers(self) -> Dimers:
        n = C.c_int64()
        self._check(self.lib.fmo_get_dimers(self.h, C.byref(n), None, None, None, None, None, None))
        m = n.value
        ij = np.zeros(2 * max(m, 1), dtype=np.int32)
        dE, ed, dev = np.zeros(max(m, 1)), np.zeros(max(m, 1)), np.zeros(max(m, 1))
        scc = np.zeros(max(m, 1), dtype=np.uint8)
        it = np.zeros(max(m, 1), dtype=np.int32)
        self._check(self.lib.fmo_get_dimers(self.h, C.byref(n), _ip(ij), _dp(dE), _dp(ed), _dp(dev),
                                            scc.ctypes.data_as(C.POINTER(C.c_uint8)), _ip(it)))
        return Dimers(ij[:2 * m].reshape(-1, 2), dE[:m], ed[:m], dev[:m], scc[:m].astype(bool), it[:m])

    def trimers(self) -> Trimers:
        n = C.c_int64()
        self._check(self.lib.fmo_get_trimers(self.h, C.byref(n), None, None, None))
        m = n.value
        ijk = np.zeros(3 * max(m, 1), dtype=np.int32)
        d3, cr = np.zeros(max(m, 1)), np.zeros(max(m, 1))
        self._check(self.lib.fmo_get_trimers(self.h, C.byref(n), _ip(ijk), _dp(d3), _dp(cr)))
        return Trimers(ijk[:3 * m].reshape(-1, 3), d3[:m], cr[:m])

    def gradient(self) -> np.ndarray:
        """dE/dxyz (n_atoms x 3, Eh/bohr) of the last run (fmo_get_gradient)."""
        g = np.zeros(3 * self.n_atoms)
        self._check(self.lib.fmo_get_gradient(self.h, _dp(g)))
        return g.reshape(-1, 3)

    # learned initial charges (options guess=1)
    def mlp_init(self, seed: int = 0):
        self._check(self.lib.fmo_mlp_init(self.h, seed))

    def mlp_set_weights(self, w: np.ndarray):
        w = np.ascontiguousarray(w, dtype=np.float32)
        self._check(self.lib.fmo_mlp_set_weights(self.h, w.ctypes.data_as(C.POINTER(C.c_float)), len(w)))

    def mlp_get_weights(self) -> np.ndarray:
        n = C.c_int64()
        self._check(self.lib.fmo_mlp_get_weights(self.h, None, C.byref(n)))
        w = np.zeros(n.value, dtype=np.float32)
        self._check(self.lib.fmo_mlp_get_weights(self.h, w.ctypes.data_as(C.POINTER(C.c_float)), C.byref(n)))
        return w

    def mlp_predict(self) -> np.ndarray:
        ns, _ = self.sizes()
        q = np.zeros(ns)
        self._check(self.lib.fmo_mlp_predict(self.h, _dp(q)))
        return q

    def mlp_train(self, xyz_frames: np.ndarray, shell_dq: np.ndarray, epochs: int, batch_frames: int = 8,
                  lr: float = 1e-3, seed: int = 0) -> np.ndarray:
        x = np.ascontiguousarray(xyz_frames, dtype=np.float64)
        q = np.ascontiguousarray(shell_dq, dtype=np.float64)
        loss = np.zeros(epochs)
        self._check(self.lib.fmo_mlp_train(self.h, len(x), _dp(x.reshape(-1)), _dp(q.reshape(-1)), epochs,
                                           batch_frames, lr, seed, _dp(loss)))
        return loss

    def mlp_loss_grad(self, xyz_frames: np.ndarray, shell_dq: np.ndarray):
        """(loss, gradient in the flat layout of the trained weights) of the
        current model on the frames, no update (fmo_mlp_loss_grad)."""
        x = np.ascontiguousarray(xyz_frames, dtype=np.float64)
        q = np.ascontiguousarray(shell_dq, dtype=np.float64)
        loss = C.c_double(0.0)
        g = np.zeros(MLP_N_TRAINED, dtype=np.float32)
        self._check(self.lib.fmo_mlp_loss_grad(self.h, len(x), _dp(x.reshape(-1)), _dp(q.reshape(-1)), C.byref(loss),
                                               g.ctypes.data_as(C.POINTER(C.c_float))))
        return loss.value, g

    def stats(self) -> dict:
        s = FmoStats()
        self._check(self.lib.fmo_get_stats(self.h, C.byref(s)))
        return s.as_dict()
