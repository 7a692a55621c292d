"""ctypes binding of include/irlnqs.h: the same entry points, argument marshalling only.

Every array argument may be a ``torch.Tensor`` (host or CUDA) or a NumPy
array; the library detects host versus device memory itself. Streams are
``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers, or ``None``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libirlnqs.so")

LM_OK, LM_ERR_ARG, LM_ERR_SIZE, LM_ERR_OOM, LM_ERR_CUDA, LM_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
LM_ERR_CALLBACK = -6
LM_REDUCE_HOST, LM_REDUCE_DEVICE = 0, 1
IRL_OK, IRL_BREAKDOWN_INVARIANT, IRL_MAX_RESTARTS, LM_C0_TINY, LM_STATIONARY = 0, 1, 2, 3, 4
LM_FP64, LM_FP32, LM_BF16, LM_DF64 = 0, 1, 2, 3
LM_SYM_AUTO, LM_SYM_NONE, LM_SYM_HALF, LM_SYM_ELOC = 0, 1, 2, 3
LM_ARITH_DF64, LM_ARITH_FP64 = 0, 1
IRL_REORTH_FULL, IRL_REORTH_NONE = 0, 1
IRL_MODE_SHEP = 0
LM_NOALLOC_MAX_LD = 2048
LM_PROF_ONLY, LM_PROF_BUILD, LM_PROF_PENCIL, LM_PROF_LANCZOS, LM_PROF_PREP, LM_PROF_TRI = \
    0x100, 0x01, 0x02, 0x04, 0x08, 0x10
EXPORT_O, EXPORT_G, EXPORT_LNPSI, EXPORT_ELOC, EXPORT_W, EXPORT_OBAR, EXPORT_ROWS = range(7)

c_int, c_double, c_int64, c_uint64, c_vp = (ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                            ctypes.c_uint64, ctypes.c_void_p)


class lm_ctx_params(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint), ("profile", c_int), ("hbm_gbs", ctypes.c_double)]


class lm_system(ctypes.Structure):
    _fields_ = [("n_orb", c_int), ("n_alpha", c_int), ("n_beta", c_int), ("n_hidden", c_int),
                ("h", c_vp), ("eri", c_vp), ("e_core", c_double), ("build_arith", c_int)]


class lm_pencil_info(ctypes.Structure):
    _fields_ = [("n_rows", c_int64), ("n_params", c_int), ("ld", c_int), ("precision", c_int),
                ("sym", c_int), ("energy", c_double), ("grid", c_int)]


class irl_params(ctypes.Structure):
    _fields_ = [("m", c_int), ("k", c_int), ("tol", c_double), ("max_restarts", c_int),
                ("seed", c_uint64), ("sym", c_int), ("precision", c_int),
                ("deflate_null", c_int), ("v0", c_vp), ("reorth", c_int), ("mode", c_int),
                ("block", c_int)]


class irl_result(ctypes.Structure):
    _fields_ = [("lambda_", c_double), ("energy", c_double), ("lambda_gen_rq", c_double),
                ("residual", c_double), ("c0", c_double), ("status", c_int),
                ("n_matvec", c_int), ("n_restart", c_int), ("n_matvec_lowp", c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class lm_batch_item(ctypes.Structure):
    _fields_ = [("sys", lm_system), ("theta", c_vp), ("rows", c_vp), ("weights", c_vp),
                ("n_rows", c_int64), ("precision", c_int), ("irl", irl_params),
                ("dtheta_out", c_vp), ("theta_inout", c_vp)]


class lm_response(ctypes.Structure):
    _fields_ = [("ticket", c_int64), ("system_id", c_int), ("status", c_int), ("grid", c_int),
                ("result", irl_result), ("t_submit_ms", c_double), ("t_admit_ms", c_double),
                ("t_done_ms", c_double)]


class lm_stats(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("build_ms", c_double), ("build_count", c_int64),
                ("pencil_ms", c_double), ("pencil_count", c_int64), ("pencil_rows", c_int64),
                ("lanczos_ms", c_double), ("lanczos_count", c_int64), ("prep_ms", c_double),
                ("prep_count", c_int64), ("tri_ms", c_double), ("tri_count", c_int64)]


# int reduce(double *vec, int n, void *stream, void *user)
REDUCE_FN = ctypes.CFUNCTYPE(c_int, c_vp, c_int, c_vp, c_vp)

_lib = None

_SIGNATURES = {
    "lm_create": (c_int, [ctypes.POINTER(c_vp), c_int, c_vp]),
    "lm_destroy": (c_int, [c_vp]),
    "lm_last_error": (ctypes.c_char_p, [c_vp]),
    "lm_build_OG": (c_int, [c_vp, ctypes.POINTER(lm_system), c_vp, c_vp, c_vp, c_int64, c_int,
                            c_vp, ctypes.POINTER(c_vp)]),
    "lm_build_O": (c_int, [c_vp, ctypes.POINTER(lm_system), c_vp, c_vp, c_vp, c_int64, c_int,
                            c_vp, ctypes.POINTER(c_vp)]),
    "lm_apply_pencil": (c_int, [c_vp, c_vp, c_vp, c_vp, c_int, c_int, c_vp]),
    "irl_step": (c_int, [c_vp, ctypes.POINTER(irl_params), ctypes.POINTER(irl_result), c_vp,
                         c_vp, c_vp, c_vp]),
    "lm_pencil_info_get": (c_int, [c_vp, ctypes.POINTER(lm_pencil_info)]),
    "lm_pencil_free": (c_int, [c_vp]),
    "lm_enumerate_sector": (c_int, [c_vp, c_int, c_int, c_int, c_vp, c_int64,
                                    ctypes.POINTER(c_int64)]),
    "lm_debug_connections": (c_int, [c_vp, ctypes.POINTER(lm_system), c_vp, c_int64, c_int, c_vp,
                                     c_vp, c_vp, c_vp]),
    "lm_pencil_export": (c_int, [c_vp, c_int, c_vp, c_vp]),
    "lm_apply_pencil_noalloc": (c_int, [c_vp, c_vp, c_vp, c_int64, c_int, c_int, c_vp, c_vp, c_vp,
                                        c_int, c_vp]),
    "lm_pencil_set_grid": (c_int, [c_vp, c_int]),
    "lm_batch_create": (c_int, [c_vp, c_int, c_int, ctypes.POINTER(c_vp)]),
    "lm_batch_run": (c_int, [c_vp, c_int, c_vp, c_vp, c_vp]),
    "lm_batch_free": (c_int, [c_vp]),
    "lm_server_create": (c_int, [c_vp, ctypes.c_size_t, c_int, c_int, ctypes.POINTER(c_vp)]),
    "lm_server_add_system": (c_int, [c_vp, ctypes.POINTER(lm_system), c_vp, c_vp, c_int64, c_int,
                                     ctypes.POINTER(c_int)]),
    "lm_server_submit": (c_int, [c_vp, c_int, c_vp, ctypes.POINTER(irl_params), c_vp,
                                 ctypes.POINTER(c_int64)]),
    "lm_server_poll": (c_int, [c_vp, c_vp, c_int, ctypes.POINTER(c_int)]),
    "lm_server_pending": (c_int, [c_vp, ctypes.POINTER(c_int)]),
    "lm_server_free": (c_int, [c_vp]),
    "lm_irl_history": (c_int, [c_vp, c_vp, c_vp, c_vp, c_int, ctypes.POINTER(c_int)]),
    "lm_debug_wait_timeout": (c_int, [c_vp, c_int, c_int64]),
    "lm_build_streamed": (c_int, [c_vp, ctypes.POINTER(lm_system), c_vp, c_vp, c_vp, c_int64,
                                  c_int64, c_int, c_vp, ctypes.POINTER(c_vp)]),
    "lm_apply_pencil_block": (c_int, [c_vp, c_vp, c_int, c_int, c_vp, c_vp, c_int, c_vp]),
    "lm_debug_pencil_block": (c_int, [c_vp, c_vp, c_int, c_int, c_vp, c_vp, c_int, c_vp,
                                      ctypes.c_uint, ctypes.c_uint, c_vp]),
    "lm_shard_build": (c_int, [c_vp, ctypes.POINTER(lm_system), c_vp, c_vp, c_vp, c_int64, c_int,
                               c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(c_double)]),
    "lm_shard_sums": (c_int, [c_vp, c_double, c_vp, c_vp]),
    "lm_shard_centre": (c_int, [c_vp, c_vp, c_vp]),
    "irl_step_sharded": (c_int, [c_vp, ctypes.POINTER(irl_params), REDUCE_FN, c_vp, c_int,
                                 ctypes.POINTER(irl_result), c_vp, c_vp, c_vp, c_vp]),
    "lm_stats_reset": (c_int, [c_vp, c_int]),
    "lm_stats_get": (c_int, [c_vp, ctypes.POINTER(lm_stats)]),
}


def lib():
    """Load libirlnqs.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


def ptr(x):
    """Raw pointer of a tensor / array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if isinstance(x, int):
        return x
    raise TypeError(f"cannot take a pointer of {type(x)}")


def stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class LMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def apply_pencil_noalloc(O_c, G_c, w, n_rows, ld, p1, v, Hv=None, Sv=None, sym=LM_SYM_NONE,
                         stream=None):
    """lm_apply_pencil_noalloc: returns the status code (device arrays only)."""
    return lib().lm_apply_pencil_noalloc(ptr(O_c), ptr(G_c), ptr(w), int(n_rows), int(ld),
                                         int(p1), ptr(v), ptr(Hv), ptr(Sv), int(sym),
                                         stream_handle(stream))


class Context:
    """lm_create / lm_destroy."""

    def __init__(self, device: int = 0, profile: bool = False, hbm_gbs: float = 0.0):
        h = c_vp()
        prm = lm_ctx_params(ctypes.sizeof(lm_ctx_params), int(profile), float(hbm_gbs))
        rc = lib().lm_create(ctypes.byref(h), device, ctypes.byref(prm))
        if rc != LM_OK:
            raise LMError(rc, f"lm_create(device={device}) failed")
        self.handle = h

    def check(self, rc, what):
        if rc != LM_OK:
            raise LMError(rc, f"{what}: {lib().lm_last_error(self.handle).decode()}")

    def close(self):
        if self.handle:
            lib().lm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def system(self, n_orb, n_alpha, n_beta, n_hidden, h, eri, e_core=0.0, arith=LM_ARITH_DF64):
        s = lm_system(n_orb, n_alpha, n_beta, n_hidden, ptr(h), ptr(eri), e_core, int(arith))
        s._keep = (h, eri)
        return s

    def build_OG(self, sys, theta, rows=None, weights=None, n_rows=0, prec=LM_FP64, stream=None,
                 pencil=None):
        """lm_build_OG; returns a Pencil (new, or the given one rebuilt in place)."""
        h = c_vp(pencil.handle if pencil is not None else None)
        if rows is not None and n_rows == 0:
            n_rows = int(rows.shape[0])
        rc = lib().lm_build_OG(self.handle, ctypes.byref(sys), ptr(theta), ptr(rows),
                               ptr(weights), int(n_rows), int(prec), stream_handle(stream),
                               ctypes.byref(h))
        self.check(rc, "lm_build_OG")
        if pencil is not None:
            return pencil
        return Pencil(self, h)

    def build_O(self, sys, theta, rows=None, weights=None, n_rows=0, prec=LM_FP64, stream=None,
                pencil=None):
        """lm_build_O: the E_loc estimator's pencil (O_c, E_loc, weights; no G'_c)."""
        h = c_vp(pencil.handle if pencil is not None else None)
        if rows is not None and n_rows == 0:
            n_rows = int(rows.shape[0])
        rc = lib().lm_build_O(self.handle, ctypes.byref(sys), ptr(theta), ptr(rows),
                              ptr(weights), int(n_rows), int(prec), stream_handle(stream),
                              ctypes.byref(h))
        self.check(rc, "lm_build_O")
        if pencil is not None:
            return pencil
        return Pencil(self, h)

    def build_streamed(self, sys, theta, chunk_rows, rows=None, weights=None, n_rows=0,
                       prec=LM_FP64, stream=None, pencil=None):
        """lm_build_streamed: a pencil whose O_c, G'_c are rebuilt chunk by chunk per product."""
        h = c_vp(pencil.handle if pencil is not None else None)
        if rows is not None and n_rows == 0:
            n_rows = int(rows.shape[0])
        rc = lib().lm_build_streamed(self.handle, ctypes.byref(sys), ptr(theta), ptr(rows),
                                     ptr(weights), int(n_rows), int(chunk_rows), int(prec),
                                     stream_handle(stream), ctypes.byref(h))
        self.check(rc, "lm_build_streamed")
        return pencil if pencil is not None else Pencil(self, h)

    def shard_build(self, sys, theta, rows, weights=None, prec=LM_FP64, stream=None,
                    pencil=None):
        """lm_shard_build: the row build of one shard; returns (Pencil, largest ln psi)."""
        h = c_vp(pencil.handle if pencil is not None else None)
        m = c_double()
        rc = lib().lm_shard_build(self.handle, ctypes.byref(sys), ptr(theta), ptr(rows),
                                  ptr(weights), int(rows.shape[0]), int(prec),
                                  stream_handle(stream), ctypes.byref(h), ctypes.byref(m))
        self.check(rc, "lm_shard_build")
        return (pencil if pencil is not None else Pencil(self, h)), m.value

    def debug_wait_timeout(self, which, limit_ns):
        """lm_debug_wait_timeout: the status code (LM_ERR_TIMEOUT when the wait gave up)."""
        return lib().lm_debug_wait_timeout(self.handle, int(which), int(limit_ns))

    def stats_reset(self, profile=False):
        """lm_stats_reset: profile False/0 counts launches only, True/1 times every kernel
        class with CUDA events, LM_PROF_ONLY | class bits (LM_PROF_BUILD, ...) only those."""
        self.check(lib().lm_stats_reset(self.handle, int(profile)), "lm_stats_reset")

    def stats(self):
        st = lm_stats()
        self.check(lib().lm_stats_get(self.handle, ctypes.byref(st)), "lm_stats_get")
        return st

    def enumerate_sector(self, n_orb, n_alpha, n_beta):
        cnt = c_int64()
        self.check(lib().lm_enumerate_sector(self.handle, n_orb, n_alpha, n_beta, None, 0,
                                             ctypes.byref(cnt)), "lm_enumerate_sector")
        out = np.zeros(cnt.value, dtype=np.uint64)
        self.check(lib().lm_enumerate_sector(self.handle, n_orb, n_alpha, n_beta, ptr(out),
                                             cnt.value, ctypes.byref(cnt)), "lm_enumerate_sector")
        return out

    def debug_connections(self, sys, rows, cap):
        rows = np.ascontiguousarray(rows, dtype=np.uint64)
        n = rows.shape[0]
        od = np.zeros((n, cap), dtype=np.uint64)
        sg = np.zeros((n, cap), dtype=np.int8)
        hv = np.zeros((n, cap))
        cnt = np.zeros(n, dtype=np.int32)
        self.check(lib().lm_debug_connections(self.handle, ctypes.byref(sys), ptr(rows), n, cap,
                                              ptr(od), ptr(sg), ptr(hv), ptr(cnt)),
                   "lm_debug_connections")
        return od, sg, hv, cnt


class Pencil:
    """Handle of a built pencil: apply, irl_step, export, info, free."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle.value if isinstance(handle, c_vp) else handle

    def info(self):
        inf = lm_pencil_info()
        self.ctx.check(lib().lm_pencil_info_get(self.handle, ctypes.byref(inf)), "info")
        return inf

    def apply(self, v, Hv=None, Sv=None, sym=LM_SYM_AUTO, prec=LM_FP64, stream=None):
        rc = lib().lm_apply_pencil(self.handle, ptr(v), ptr(Hv), ptr(Sv), int(sym), int(prec),
                                   stream_handle(stream))
        self.ctx.check(rc, "lm_apply_pencil")

    def irl_step(self, m=20, k=1, tol=1e-12, max_restarts=200, seed=111, sym=LM_SYM_AUTO,
                 prec=LM_FP64, deflate_null=1, v0=None, c_out=None, dtheta_out=None,
                 theta_inout=None, stream=None, reorth=IRL_REORTH_FULL, block=0):
        prm = irl_params(m, k, tol, max_restarts, seed, int(sym), int(prec), int(deflate_null),
                         ptr(v0), int(reorth), IRL_MODE_SHEP, int(block))
        res = irl_result()
        rc = lib().irl_step(self.handle, ctypes.byref(prm), ctypes.byref(res), ptr(c_out),
                            ptr(dtheta_out), ptr(theta_inout), stream_handle(stream))
        self.ctx.check(rc, "irl_step")
        return res

    def shard_sums(self, lnpsi_max, stream=None):
        """lm_shard_sums: this shard's P+3 sums [sum w, sum w E_loc, sum w O_0..P]."""
        out = np.zeros(self.info().n_params + 3)
        self.ctx.check(lib().lm_shard_sums(self.handle, float(lnpsi_max), ptr(out),
                                           stream_handle(stream)), "lm_shard_sums")
        return out

    def shard_centre(self, sums, stream=None):
        sums = np.ascontiguousarray(sums, dtype=np.float64)
        self.ctx.check(lib().lm_shard_centre(self.handle, ptr(sums), stream_handle(stream)),
                       "lm_shard_centre")

    def irl_step_sharded(self, reduce, where=LM_REDUCE_HOST, m=20, k=1, tol=1e-12,
                         max_restarts=200, seed=111, sym=LM_SYM_AUTO, prec=LM_FP64,
                         deflate_null=1, c_out=None, dtheta_out=None, theta_inout=None,
                         stream=None):
        """irl_step_sharded. reduce(vec, n, stream) sums the n-vector over the shards in
        place: with where = LM_REDUCE_HOST, vec is a NumPy view of pinned host memory;
        with LM_REDUCE_DEVICE, the raw device pointer (an int). Returns 0 on success."""
        def cb(vp, n, st, _user):
            try:
                if where == LM_REDUCE_HOST:
                    vec = np.ctypeslib.as_array((c_double * n).from_address(vp))
                else:
                    vec = vp
                rc = reduce(vec, n, st)
                return int(rc or 0)
            except Exception:
                return 1
        fn = REDUCE_FN(cb)
        prm = irl_params(m, k, tol, max_restarts, seed, int(sym), int(prec), int(deflate_null),
                         None, IRL_REORTH_FULL, IRL_MODE_SHEP, 0)
        res = irl_result()
        rc = lib().irl_step_sharded(self.handle, ctypes.byref(prm), fn, None, int(where),
                                    ctypes.byref(res), ptr(c_out), ptr(dtheta_out),
                                    ptr(theta_inout), stream_handle(stream))
        self.ctx.check(rc, "irl_step_sharded")
        return res

    def apply_block(self, V, HV=None, SV=None, sym=LM_SYM_AUTO, stream=None, nvec=None,
                    ldv=None):
        """lm_apply_pencil_block on device arrays: V holds nvec vectors of P+1 entries with
        stride ldv (a (nvec, ldv) row-major CUDA tensor); HV, SV likewise (either None)."""
        nvec = int(V.shape[0]) if nvec is None else int(nvec)
        ldv = int(V.shape[1]) if ldv is None else int(ldv)
        rc = lib().lm_apply_pencil_block(self.handle, ptr(V), ldv, nvec, ptr(HV), ptr(SV),
                                         int(sym), stream_handle(stream))
        self.ctx.check(rc, "lm_apply_pencil_block")

    def debug_block(self, V, HV, SV, sym, dbg, lbo_mn=16384, sbo_mn=1024, stream=None):
        rc = lib().lm_debug_pencil_block(self.handle, ptr(V), int(V.shape[1]), int(V.shape[0]),
                                         ptr(HV), ptr(SV), int(sym), ptr(dbg), int(lbo_mn),
                                         int(sbo_mn), stream_handle(stream))
        self.ctx.check(rc, "lm_debug_pencil_block")

    def irl_history(self):
        """lm_irl_history: per-cycle (lowest Ritz value, residual estimate, low-precision flag)
        of the last irl_step, as three arrays."""
        n = c_int()
        self.ctx.check(lib().lm_irl_history(self.handle, None, None, None, 0, ctypes.byref(n)),
                       "lm_irl_history")
        k = n.value
        lam, res, lowp = np.zeros(k), np.zeros(k), np.zeros(k, dtype=np.int32)
        self.ctx.check(lib().lm_irl_history(self.handle, ptr(lam), ptr(res), ptr(lowp), k,
                                            ctypes.byref(n)), "lm_irl_history")
        return lam, res, lowp

    def export(self, what, out=None):
        inf = self.info()
        if out is None:
            if what in (EXPORT_O, EXPORT_G):
                out = np.zeros((inf.n_rows, inf.ld))
            elif what == EXPORT_OBAR:
                out = np.zeros(inf.ld)
            elif what == EXPORT_ROWS:
                out = np.zeros(inf.n_rows, dtype=np.uint64)
            else:
                out = np.zeros(inf.n_rows)
        self.ctx.check(lib().lm_pencil_export(self.handle, int(what), ptr(out), None), "export")
        return out

    def set_grid(self, ctas):
        self.ctx.check(lib().lm_pencil_set_grid(self.handle, int(ctas)), "lm_pencil_set_grid")

    def free(self):
        if self.handle:
            lib().lm_pencil_free(self.handle)
            self.handle = None


def irl_settings(m=20, k=1, tol=1e-12, max_restarts=200, seed=111, sym=LM_SYM_AUTO,
                 prec=LM_FP64, deflate_null=1, reorth=IRL_REORTH_FULL):
    return irl_params(m, k, tol, max_restarts, seed, int(sym), int(prec), int(deflate_null), None,
                      int(reorth), IRL_MODE_SHEP, 0)


class Batch:
    """lm_batch_create / lm_batch_run / lm_batch_free."""

    def __init__(self, ctx: Context, n_streams=16, autotune=True):
        h = c_vp()
        ctx.check(lib().lm_batch_create(ctx.handle, int(n_streams), int(autotune),
                                        ctypes.byref(h)), "lm_batch_create")
        self.ctx, self.handle = ctx, h.value

    def run(self, items):
        """items: list of dicts with sys, theta, rows, weights, n_rows, precision, irl
        (an irl_params), dtheta_out, theta_inout. Returns (results, grids)."""
        n = len(items)
        arr = (lm_batch_item * n)()
        keep = []
        for i, it in enumerate(items):
            rows = it.get("rows")
            arr[i].sys = it["sys"]
            arr[i].theta = ptr(it["theta"])
            arr[i].rows = ptr(rows)
            arr[i].weights = ptr(it.get("weights"))
            arr[i].n_rows = int(it.get("n_rows", 0 if rows is None else rows.shape[0]))
            arr[i].precision = int(it.get("precision", LM_FP32))
            arr[i].irl = it["irl"]
            arr[i].dtheta_out = ptr(it.get("dtheta_out"))
            arr[i].theta_inout = ptr(it.get("theta_inout"))
            keep.append(it)
        res = (irl_result * n)()
        grids = (c_int * n)()
        rc = lib().lm_batch_run(self.handle, n, ctypes.cast(arr, c_vp), ctypes.cast(res, c_vp),
                                ctypes.cast(grids, c_vp))
        self.ctx.check(rc, "lm_batch_run")
        return list(res), list(grids)

    def free(self):
        if self.handle:
            lib().lm_batch_free(self.handle)
            self.handle = None


class Server:
    """lm_server_*: submit LM-step requests, poll for finished responses."""

    def __init__(self, ctx: Context, hbm_budget_bytes, n_streams=16, autotune=True):
        h = c_vp()
        ctx.check(lib().lm_server_create(ctx.handle, int(hbm_budget_bytes), int(n_streams),
                                         int(autotune), ctypes.byref(h)), "lm_server_create")
        self.ctx, self.handle = ctx, h.value

    def add_system(self, sys, rows=None, weights=None, precision=LM_FP32):
        sid = c_int()
        n = 0 if rows is None else int(rows.shape[0])
        self.ctx.check(lib().lm_server_add_system(self.handle, ctypes.byref(sys), ptr(rows),
                                                  ptr(weights), n, int(precision),
                                                  ctypes.byref(sid)), "lm_server_add_system")
        return sid.value

    def submit(self, system_id, theta, irl, dtheta_out=None):
        t = c_int64()
        self.ctx.check(lib().lm_server_submit(self.handle, int(system_id), ptr(theta),
                                              ctypes.byref(irl), ptr(dtheta_out),
                                              ctypes.byref(t)), "lm_server_submit")
        return t.value

    def poll(self, cap=64):
        buf = (lm_response * cap)()
        n = c_int()
        self.ctx.check(lib().lm_server_poll(self.handle, ctypes.cast(buf, c_vp), cap,
                                            ctypes.byref(n)), "lm_server_poll")
        return [buf[i] for i in range(n.value)]

    def pending(self):
        n = c_int()
        self.ctx.check(lib().lm_server_pending(self.handle, ctypes.byref(n)), "pending")
        return n.value

    def free(self):
        if self.handle:
            lib().lm_server_free(self.handle)
            self.handle = None
