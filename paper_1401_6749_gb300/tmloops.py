"""Thin ctypes binding of the tmloops C ABI (include/tmloops.h).

Argument marshalling only: every function forwards to the entry point of the
same name in libtmloops.so; tensors are passed by device pointer, the stream
defaults to torch's current stream.  Importing this module loads the library
and raises if it is missing — there is no fallback path.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtmloops.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libtmloops.so is not built; run paper_1401_6749_gb300.build.build() "
                      "(or __graft_entry__.build()) first")
_lib = ctypes.CDLL(LIB_PATH)

# precisions, modes, status codes (tmloops.h)
F64, F32, F16, BF16, FF = 0, 1, 2, 3, 4
PREC = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16, "ff": FF}
CG_PLAIN, CG_MIXED = 0, 1
LOOP_STD, LOOP_VV, LOOP_GEN = 0, 1, 2
LOOP_MODE = {"std": LOOP_STD, "vv": LOOP_VV, "gen": LOOP_GEN}
STATUS = {0: "TM_OK", 1: "TM_ERR_ARG", 2: "TM_ERR_CUDA", 3: "TM_ERR_NOCONV", 4: "TM_ERR_NAN",
          5: "TM_ERR_TIMEOUT", 6: "TM_ERR_UNSUPPORTED"}
ELEM_SIZE = {F64: 8, F32: 4, F16: 2, BF16: 2, FF: 8}


class TmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class tm_geom_t(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4)]


class tm_params_t(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("kappa", ctypes.c_double), ("mu", ctypes.c_double),
                ("antiperiodic_t", ctypes.c_int), ("recon", ctypes.c_int)]


class tm_cg_params_t(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mode", ctypes.c_int),
                ("prec", ctypes.c_int), ("inner_prec", ctypes.c_int), ("delta", ctypes.c_double),
                ("check_every", ctypes.c_int), ("true_residual", ctypes.c_int), ("schur", ctypes.c_int),
                ("graph", ctypes.c_int), ("ru_prec", ctypes.c_int)]


class tm_cg_stats_t(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("status", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("true_res", ctypes.c_double)]


_vp, _i, _d, _u32, _u64, _sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint32,
                                ctypes.c_uint64, ctypes.c_size_t)
_P = ctypes.POINTER
_SIGS = {
    "tm_op_create": [_P(_vp), _P(tm_params_t), _vp, _vp],
    "tm_op_destroy": [_vp],
    "tm_op_clone": [_P(_vp), _vp],
    "tm_mem_trim": [_sz],
    "tm_dslash_mma_enable": [_i],
    "tm_mem_reserved": [_P(_sz)],
    "tm_spinor_bytes": [_P(tm_geom_t), _i, _i],
    "tm_spinor_pack": [_P(tm_geom_t), _vp, _i, _vp, _i, _vp],
    "tm_spinor_unpack": [_P(tm_geom_t), _vp, _vp, _i, _i, _vp],
    "tm_spinor_convert": [_P(tm_geom_t), _vp, _i, _vp, _i, _i, _vp],
    "tm_gamma5": [_P(tm_geom_t), _vp, _vp, _i, _i, _vp],
    "tm_dslash": [_vp, _vp, _vp, _i, _i, _i, _i, _vp],
    "tm_dslash_g5": [_vp, _vp, _vp, _i, _i, _i, _i, _vp],
    "z4_noise": [_P(tm_geom_t), _vp, _i, _u64, _u32, _i, _vp],
    "tm_cg_solve": [_vp, _vp, _vp, _i, _P(tm_cg_params_t), _P(tm_cg_stats_t), _vp],
    "tm_cg_solve_group": [_i, _P(_vp), _P(_vp), _P(_vp), _P(_i), _P(tm_cg_params_t), _P(_P(tm_cg_stats_t)),
                          _vp],
    "loop_contract_local": [_P(tm_geom_t), _vp, _vp, _i, _i, _i, _vp, _vp],
    "loop_contract_oneD": [_vp, _vp, _vp, _i, _i, _i, _vp, _vp],
    "loop_contract_local_noalloc": [_P(tm_geom_t), _vp, _vp, _i, _i, _i, _vp, _vp],
    "tsm_combine": [_vp, _vp, _i, _vp, _i, _sz, _d, _d, _vp, _vp, _vp],
    "z4_noise_diluted": [_P(tm_geom_t), _vp, _i, _u64, _u32, _i, _i, _i, _vp],
    "z4_noise_il": [_P(tm_geom_t), _vp, _i, _u64, _u32, _i, _vp],
    "tm_hpe_apply": [_vp, _vp, _vp, _i, _i, _i, _vp],
    "tm_hpe_exact": [_P(tm_params_t), _vp],
    "loop_contract_local_mom": [_P(tm_geom_t), _vp, _vp, _i, _i, _i, _vp, _i, _vp, _vp],
    "tm_last_error": [],
    "tm_launch_count": [],
    "tm_trace_enable": [_i],
    "tm_trace_reset": [],
    "tm_trace_read": [ctypes.c_char_p, _P(_i), _P(_d), _P(_d)],
    "tm_trace_read_flops": [ctypes.c_char_p, _P(_d)],
    "tm_tune_enable": [_i],
    "tm_tune_reset": [],
    "tm_tune_count": [],
    "tm_tune_get": [_i, _P(_i), _P(_i), _P(_i), _P(_i)],
    "tm_spinor_bytes_il": [_P(tm_geom_t), _i],
    "tm_spinor_to_il": [_P(tm_geom_t), _vp, _vp, _i, _i, _vp],
    "tm_spinor_from_il": [_P(tm_geom_t), _vp, _vp, _i, _i, _vp],
    "tm_dslash_il": [_vp, _vp, _vp, _i, _i, _i, _i, _vp],
    "tm_cg_il_enable": [_i],
    "tm_op_check": [_vp],
    "tsm_combine_host": [_vp, _vp, _i, _vp, _i, _sz, _d, _d, _vp, _vp],
    "tm_cg_solve_il": [_vp, _vp, _vp, _i, _P(tm_cg_params_t), _P(tm_cg_stats_t), _vp],
    "loop_contract_local_il": [_P(tm_geom_t), _vp, _vp, _i, _i, _i, _i, _vp, _vp],
    "loop_contract_oneD_il": [_vp, _vp, _vp, _i, _i, _i, _i, _vp, _vp],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _i
_lib.tm_spinor_bytes.restype = _sz
_lib.tm_spinor_bytes_il.restype = _sz
_lib.tm_last_error.restype = ctypes.c_char_p
_lib.tm_launch_count.restype = _u64
_lib.tm_trace_enable.restype = None
_lib.tm_trace_reset.restype = None
_lib.tm_tune_enable.restype = None
_lib.tm_tune_reset.restype = None

EXPORTED = tuple(_SIGS)


def _check(status):
    if status != 0:
        raise TmError(status, _lib.tm_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def geom(L):
    g = tm_geom_t()
    for i in range(4):
        g.L[i] = int(L[i])
    return g


def tm_spinor_bytes(L, prec, nrhs):
    return int(_lib.tm_spinor_bytes(ctypes.byref(geom(L)), int(prec), int(nrhs)))


def empty_field(L, prec, nrhs, device="cuda"):
    """Uninitialised internal-layout field storage (uint8 tensor, 256-byte aligned)."""
    return torch.empty(tm_spinor_bytes(L, prec, nrhs), dtype=torch.uint8, device=device)


def link_reals(recon, prec):
    """Reals stored per link in the operator's copy of precision prec
    (recon 0 = per precision: 12 for F32, 18 for F16/BF16; F64 always 18)."""
    if prec in (F64, FF):
        return 18
    if recon == 0:
        return 12 if prec == F32 else 18
    return int(recon)


class Operator:
    """Owner of a tm_op_t handle (gauge links in every precision).  U: the FP64
    lexicographic gauge field as a CUDA tensor or a pinned CPU tensor (read by
    the GPU directly)."""

    def __init__(self, L, kappa, mu, U, antiperiodic=True, recon=12, stream=None):
        self.L = tuple(int(v) for v in L)
        self.kappa, self.mu = float(kappa), float(mu)
        self.recon = int(recon)
        p = tm_params_t()
        for i in range(4):
            p.L[i] = self.L[i]
        p.kappa, p.mu, p.antiperiodic_t, p.recon = self.kappa, self.mu, int(bool(antiperiodic)), int(recon)
        h = ctypes.c_void_p()
        _check(_lib.tm_op_create(ctypes.byref(h), ctypes.byref(p), _ptr(U), _stream(stream)))
        self.handle = h

    def clone(self):
        """Handle sharing these links with its own solver work space (for a
        concurrent solve on another thread and stream); close it before self."""
        c = Operator.__new__(Operator)
        c.L, c.kappa, c.mu, c.recon = self.L, self.kappa, self.mu, self.recon
        h = ctypes.c_void_p()
        _check(_lib.tm_op_clone(ctypes.byref(h), self.handle))
        c.handle = h
        c._source = self  # keeps the link owner alive
        return c

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.tm_op_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tm_dslash_mma_enable(on=True):
    """Run the FP16/BF16 18-real-link Dslash on the tensor cores (or not)."""
    _check(_lib.tm_dslash_mma_enable(int(bool(on))))


def tm_mem_trim(keep_bytes=0):
    """Release unused memory of the library's device pool beyond keep_bytes."""
    _check(_lib.tm_mem_trim(int(keep_bytes)))


def tm_mem_reserved():
    """Bytes held by the library's device pool on the current device."""
    v = ctypes.c_size_t()
    _check(_lib.tm_mem_reserved(ctypes.byref(v)))
    return v.value


def tm_spinor_pack(L, out, prec, in_lex, nrhs, stream=None):
    _check(_lib.tm_spinor_pack(ctypes.byref(geom(L)), _ptr(out), int(prec), _ptr(in_lex), int(nrhs),
                               _stream(stream)))


def tm_spinor_unpack(L, out_lex, inp, prec, nrhs, stream=None):
    _check(_lib.tm_spinor_unpack(ctypes.byref(geom(L)), _ptr(out_lex), _ptr(inp), int(prec), int(nrhs),
                                 _stream(stream)))


def tm_spinor_convert(L, out, out_prec, inp, in_prec, nrhs, stream=None):
    _check(_lib.tm_spinor_convert(ctypes.byref(geom(L)), _ptr(out), int(out_prec), _ptr(inp),
                                  int(in_prec), int(nrhs), _stream(stream)))


def tm_gamma5(L, out, inp, prec, nrhs, stream=None):
    _check(_lib.tm_gamma5(ctypes.byref(geom(L)), _ptr(out), _ptr(inp), int(prec), int(nrhs),
                          _stream(stream)))


def tm_dslash(op, out, inp, nrhs, dagger=False, mu_zero=False, prec=F32, stream=None):
    _check(_lib.tm_dslash(op.handle, _ptr(out), _ptr(inp), int(nrhs), int(bool(dagger)),
                          int(bool(mu_zero)), int(prec), _stream(stream)))


def tm_spinor_bytes_il(L, nrhs):
    return int(_lib.tm_spinor_bytes_il(ctypes.byref(geom(L)), int(nrhs)))


def empty_field_il(L, nrhs, device="cuda"):
    """Uninitialised storage of nrhs 16-bit fields in the system-interleaved layout."""
    return torch.empty(tm_spinor_bytes_il(L, nrhs), dtype=torch.uint8, device=device)


def z4_noise_il(L, eta_il, prec, seed, first_src, nsrc, stream=None):
    """z4_noise written straight into the interleaved layout (F16 or BF16)."""
    _check(_lib.z4_noise_il(ctypes.byref(geom(L)), _ptr(eta_il), int(prec), int(seed), int(first_src),
                            int(nsrc), _stream(stream)))


def tm_spinor_to_il(L, out_il, inp, prec, nrhs, stream=None):
    _check(_lib.tm_spinor_to_il(ctypes.byref(geom(L)), _ptr(out_il), _ptr(inp), int(prec), int(nrhs),
                                _stream(stream)))


def tm_spinor_from_il(L, out, inp_il, prec, nrhs, stream=None):
    _check(_lib.tm_spinor_from_il(ctypes.byref(geom(L)), _ptr(out), _ptr(inp_il), int(prec), int(nrhs),
                                  _stream(stream)))


def tm_dslash_il(op, out_il, inp_il, nrhs, dagger=False, mu_zero=False, prec=F16, stream=None):
    """M (M^dag, D_W) on 16-bit fields in the system-interleaved layout (tensor cores)."""
    _check(_lib.tm_dslash_il(op.handle, _ptr(out_il), _ptr(inp_il), int(nrhs), int(bool(dagger)),
                             int(bool(mu_zero)), int(prec), _stream(stream)))


def tm_op_check(op):
    """Wait for the device; raise TM_ERR_TIMEOUT if a bounded wait of a kernel
    on this operator gave up since the last check."""
    _check(_lib.tm_op_check(op.handle))


def tm_cg_il_enable(on=True):
    """Plain F16/BF16 solves on the interleaved layout (default) or the standard one."""
    _check(_lib.tm_cg_il_enable(int(bool(on))))


def tm_dslash_g5(op, out, inp, nrhs, dagger=False, mu_zero=False, prec=F32, stream=None):
    """out = gamma_5 (M, M^dag or D_W) inp in one pass."""
    _check(_lib.tm_dslash_g5(op.handle, _ptr(out), _ptr(inp), int(nrhs), int(bool(dagger)),
                             int(bool(mu_zero)), int(prec), _stream(stream)))


def z4_noise(L, eta, prec, seed, first_src, nsrc, stream=None):
    _check(_lib.z4_noise(ctypes.byref(geom(L)), _ptr(eta), int(prec), int(seed), int(first_src),
                         int(nsrc), _stream(stream)))


def cg_params(tol, max_iter=10000, mode=CG_PLAIN, prec=F64, inner_prec=F32, delta=0.1,
              check_every=8, true_residual=False, schur=False, graph=False, ru_prec=F64):
    p = tm_cg_params_t()
    p.tol, p.max_iter, p.mode, p.prec, p.inner_prec = float(tol), int(max_iter), int(mode), int(prec), int(inner_prec)
    p.delta, p.check_every, p.true_residual = float(delta), int(check_every), int(bool(true_residual))
    p.schur, p.graph, p.ru_prec = int(bool(schur)), int(bool(graph)), int(ru_prec)
    return p


def tm_cg_solve(op, x, eta, nrhs, params, stream=None, raise_on_noconv=True):
    """Returns (status, list of per-system dicts).  raise_on_noconv=False returns
    the per-system solver outcomes TM_ERR_NOCONV and TM_ERR_NAN with the stats
    instead of raising (argument and CUDA errors always raise)."""
    stats = (tm_cg_stats_t * max(int(nrhs), 1))()
    st = _lib.tm_cg_solve(op.handle, _ptr(x), _ptr(eta), int(nrhs), ctypes.byref(params), stats,
                          _stream(stream))
    out = [dict(iters=s.iters, reliable_updates=s.reliable_updates, status=s.status,
                rel_res=s.rel_res, true_res=s.true_res) for s in list(stats)[:int(nrhs)]]
    if st != 0 and (st not in (3, 4) or raise_on_noconv):
        _check(st)
    return st, out


def tm_cg_solve_il(op, x_il, eta_il, nrhs, params, stream=None, raise_on_noconv=True):
    """tm_cg_solve with sources and solutions in the interleaved layout (both
    from empty_field_il); the same return values."""
    stats = (tm_cg_stats_t * max(int(nrhs), 1))()
    st = _lib.tm_cg_solve_il(op.handle, _ptr(x_il), _ptr(eta_il), int(nrhs), ctypes.byref(params), stats,
                             _stream(stream))
    out = [dict(iters=s.iters, reliable_updates=s.reliable_updates, status=s.status,
                rel_res=s.rel_res, true_res=s.true_res) for s in list(stats)[:int(nrhs)]]
    if st != 0 and (st not in (3, 4) or raise_on_noconv):
        _check(st)
    return st, out


def tm_cg_solve_group(ops, xs, etas, nrhs, params, stream=None, raise_on_noconv=True):
    """Several solves (one per operator) advanced together; returns
    (status, [per-set list of per-system dicts])."""
    n = len(ops)
    if not (len(xs) == len(etas) == len(nrhs) == n):
        raise ValueError("ops, xs, etas and nrhs must have the same length")
    arr = lambda vals: (_vp * max(n, 1))(*vals)
    stats = [(tm_cg_stats_t * max(int(k), 1))() for k in nrhs]
    sp = (_P(tm_cg_stats_t) * max(n, 1))(*[ctypes.cast(s, _P(tm_cg_stats_t)) for s in stats])
    st = _lib.tm_cg_solve_group(n, arr([o.handle for o in ops]), arr([_ptr(x) for x in xs]),
                                arr([_ptr(e) for e in etas]), (_i * max(n, 1))(*[int(k) for k in nrhs]),
                                ctypes.byref(params), sp, _stream(stream))
    out = [[dict(iters=s.iters, reliable_updates=s.reliable_updates, status=s.status, rel_res=s.rel_res,
                 true_res=s.true_res) for s in list(ss)[:int(k)]] for ss, k in zip(stats, nrhs)]
    if st != 0 and (st not in (3, 4) or raise_on_noconv):
        _check(st)
    return st, out


def loop_contract_local(L, left, right, prec, nrhs, mode, out, stream=None):
    _check(_lib.loop_contract_local(ctypes.byref(geom(L)), _ptr(left), _ptr(right), int(prec),
                                    int(nrhs), int(mode), _ptr(out), _stream(stream)))


def loop_contract_local_noalloc(L, left, right, prec, nrhs, mode, out, stream=None):
    """loop_contract_local without device allocation (fixed 8 MiB scratch in the
    library; calls that overlap on the GPU race)."""
    _check(_lib.loop_contract_local_noalloc(ctypes.byref(geom(L)), _ptr(left), _ptr(right), int(prec),
                                            int(nrhs), int(mode), _ptr(out), _stream(stream)))


def loop_contract_oneD(op, left, right, prec, nrhs, mode, out, stream=None):
    _check(_lib.loop_contract_oneD(op.handle, _ptr(left), _ptr(right), int(prec), int(nrhs), int(mode),
                                   _ptr(out), _stream(stream)))


def loop_contract_local_il(L, left_il, right_il, prec, nrhs, mode, out, right_g5=False, stream=None):
    """Local loops of fields in the interleaved layout (right_g5: R = gamma_5 right_il)."""
    _check(_lib.loop_contract_local_il(ctypes.byref(geom(L)), _ptr(left_il), _ptr(right_il), int(prec),
                                       int(nrhs), int(mode), int(bool(right_g5)), _ptr(out), _stream(stream)))


def loop_contract_oneD_il(op, left_il, right_il, prec, nrhs, mode, out, right_g5=False, stream=None):
    """One-derivative loops of fields in the interleaved layout (tensor cores;
    right_g5: R = gamma_5 right_il)."""
    _check(_lib.loop_contract_oneD_il(op.handle, _ptr(left_il), _ptr(right_il), int(prec), int(nrhs),
                                      int(mode), int(bool(right_g5)), _ptr(out), _stream(stream)))


def tsm_combine(l_hp, l_lp_on_hp, n_hp, l_lp, n_lp, length, scale, mean, err, stream=None):
    scale = complex(scale)
    _check(_lib.tsm_combine(_ptr(l_hp), _ptr(l_lp_on_hp), int(n_hp), _ptr(l_lp), int(n_lp),
                            int(length), scale.real, scale.imag, _ptr(mean), _ptr(err), _stream(stream)))


def tsm_combine_host(l_hp, l_lp_on_hp, n_hp, l_lp, n_lp, length, scale, mean, err):
    """Eq. 4 on host (CPU) float64 tensors; synchronous."""
    for t in (l_hp, l_lp_on_hp, l_lp, mean, err):
        if t is not None and (t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous()):
            raise ValueError("tsm_combine_host takes contiguous float64 host tensors")
    sc = complex(scale)
    _check(_lib.tsm_combine_host(_ptr(l_hp), _ptr(l_lp_on_hp), int(n_hp), _ptr(l_lp), int(n_lp),
                                 int(length), sc.real, sc.imag, _ptr(mean), _ptr(err)))


def z4_noise_diluted(L, eta, prec, seed, first_src, nsrc, t0, dt, stream=None):
    _check(_lib.z4_noise_diluted(ctypes.byref(geom(L)), _ptr(eta), int(prec), int(seed), int(first_src),
                                 int(nsrc), int(t0), int(dt), _stream(stream)))


def tm_hpe_apply(op, out, inp, nrhs, order, prec, stream=None):
    _check(_lib.tm_hpe_apply(op.handle, _ptr(out), _ptr(inp), int(nrhs), int(order), int(prec),
                             _stream(stream)))


def tm_hpe_exact(L, kappa, mu, antiperiodic=True):
    """Exact HPE part of the local loops: numpy complex (16, T) (host computation)."""
    import numpy as np
    p = tm_params_t()
    for i in range(4):
        p.L[i] = int(L[i])
    p.kappa, p.mu, p.antiperiodic_t, p.recon = float(kappa), float(mu), int(bool(antiperiodic)), 18
    out = np.zeros((16, int(L[3]), 2), dtype=np.float64)
    _check(_lib.tm_hpe_exact(ctypes.byref(p), out.ctypes.data_as(ctypes.c_void_p)))
    return out[..., 0] + 1j * out[..., 1]


def loop_contract_local_mom(L, left, right, prec, nrhs, mode, momenta, out, stream=None):
    import numpy as np
    mom = np.ascontiguousarray(np.asarray(momenta, dtype=np.int32).reshape(-1, 3))
    _check(_lib.loop_contract_local_mom(ctypes.byref(geom(L)), _ptr(left), _ptr(right), int(prec),
                                        int(nrhs), int(mode), mom.ctypes.data_as(ctypes.c_void_p),
                                        int(mom.shape[0]), _ptr(out), _stream(stream)))


def tm_launch_count():
    return int(_lib.tm_launch_count())


def tm_trace_enable(on):
    _lib.tm_trace_enable(int(bool(on)))


def tm_trace_reset():
    _lib.tm_trace_reset()


def tm_trace_read(name="dslash.*"):
    """(launches, device ms, algorithmic bytes) of a traced Dslash class."""
    n = ctypes.c_int()
    ms = ctypes.c_double()
    nb = ctypes.c_double()
    _check(_lib.tm_trace_read(name.encode(), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(nb)))
    return n.value, ms.value, nb.value


def tm_trace_read_flops(name="dslash.*"):
    """Algorithmic flops of a traced Dslash class (same launches as tm_trace_read)."""
    f = ctypes.c_double()
    _check(_lib.tm_trace_read_flops(name.encode(), ctypes.byref(f)))
    return f.value


def tm_tune_enable(on):
    _lib.tm_tune_enable(int(bool(on)))


def tm_tune_reset():
    _lib.tm_tune_reset()


def tm_tune_entries():
    """The autotuner's choices: list of (key dict, systems per thread, block size,
    packed FP32x2 flag)."""
    out = []
    names = ("prec", "link_reals", "dagger", "epilogue", "parity", "centre", "out_inv", "half_volume", "nrhs")
    for i in range(_lib.tm_tune_count()):
        key = (_i * 9)()
        nr, bx, pk = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.tm_tune_get(i, key, ctypes.byref(nr), ctypes.byref(bx), ctypes.byref(pk)))
        out.append((dict(zip(names, list(key))), nr.value, bx.value, pk.value))
    return out
