"""ctypes binding of libdsd (include/dsd.h).

Argument marshalling only: every computation runs in the CUDA library.
The module-level ``dsd_*`` functions mirror the C entry points one to one
(pointers are passed as integers); :class:`Graph` is a thin convenience
wrapper that allocates outputs as numpy arrays (host) or torch CUDA tensors
(device).  If the compiled library is missing, importing the wrappers raises
an error -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdsd.so")

DSD_MEM_HOST = 0
DSD_MEM_DEVICE = 1
DSD_PATTERN_STAR = 1
DSD_PATTERN_LOOP4 = 2
DSD_NPHASES = 6
PHASES = ("csr", "order_peel", "orient", "count", "peel", "extract")

STATUS = {0: "DSD_OK", 1: "DSD_ERR_INVALID", 2: "DSD_ERR_NOMEM", 3: "DSD_ERR_CUDA",
          4: "DSD_ERR_TIMEOUT", 5: "DSD_ERR_OVERFLOW", 6: "DSD_ERR_INTERNAL",
          7: "DSD_ERR_UNSUPPORTED"}


class DSDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status
        self.name = STATUS.get(status, str(status))


class CoreAppResult(ctypes.Structure):
    _fields_ = [("kmax", ctypes.c_uint64), ("kmax_core_size", ctypes.c_uint32),
                ("densest_size", ctypes.c_uint32), ("kmax_core_mu", ctypes.c_uint64),
                ("best_k", ctypes.c_uint64), ("densest_mu", ctypes.c_uint64),
                ("nlevels", ctypes.c_uint32), ("seeded_accepted", ctypes.c_int32),
                ("seed_k", ctypes.c_uint64)]


class PeelAppResult(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_uint64), ("size", ctypes.c_uint32),
                ("removed", ctypes.c_uint32), ("level_k", ctypes.c_uint64)]


class TopdownInfo(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_uint32), ("sub_n", ctypes.c_uint32), ("x", ctypes.c_uint64),
                ("gamma_out", ctypes.c_uint64), ("sub_m", ctypes.c_uint64)]


class ExactInfo(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_uint64), ("size", ctypes.c_uint32), ("cuts", ctypes.c_uint32),
                ("k1", ctypes.c_uint64), ("k2", ctypes.c_uint64), ("lower_mu", ctypes.c_uint64),
                ("lower_size", ctypes.c_uint32), ("components", ctypes.c_uint32),
                ("net_nodes", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("net_arcs", ctypes.c_uint64), ("rounds", ctypes.c_uint64),
                ("relabels", ctypes.c_uint64), ("locate_ns", ctypes.c_uint64),
                ("build_ns", ctypes.c_uint64), ("cut_ns", ctypes.c_uint64),
                ("verify_ns", ctypes.c_uint64)]


class SeedInfo(ctypes.Structure):
    _fields_ = [("rho_prime", ctypes.c_float), ("accepted", ctypes.c_uint32),
                ("seed_k", ctypes.c_uint64), ("x0", ctypes.c_uint64),
                ("sub_n", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("sub_m", ctypes.c_uint64)]


NFEAT = 64

_lib = None

_P = ctypes.c_void_p
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_int = ctypes.c_int

SIGNATURES = {
    "dsd_status_string": (ctypes.c_char_p, [_int]),
    "dsd_last_error": (ctypes.c_char_p, []),
    "dsd_version": (ctypes.c_char_p, []),
    "dsd_kernel_launches": (ctypes.c_uint64, []),
    "dsd_set_wait_limit_ms": (_int, [_u32]),
    "dsd_set_peel_small_limit": (_int, [_u32]),
    "dsd_set_peel_tail_limit": (_int, [_u32]),
    "dsd_set_peel_app_queue": (_int, [_u32, ctypes.c_uint64]),
    "dsd_set_peel_items": (_int, [_u32, _u32]),
    "dsd_graph_from_edges": (_int, [_u32, _u64, _P, _P, _int, _P, ctypes.POINTER(_P)]),
    "dsd_graph_from_csr": (_int, [_u32, _P, _P, _int, _P, ctypes.POINTER(_P)]),
    "dsd_graph_destroy": (None, [_P]),
    "dsd_graph_info": (_int, [_P, _P, _P]),
    "dsd_graph_set_stream": (_int, [_P, _P]),
    "dsd_graph_csr": (_int, [_P, _P, _P, _int]),
    "dsd_degeneracy_order": (_int, [_P, _P, _P, _P, _int]),
    "dsd_clique_degrees": (_int, [_P, _int, _P, _P, _int]),
    "dsd_core_decompose": (_int, [_P, _int, _P, _P, _int]),
    "dsd_level_stats": (_int, [_P, _int, _P, _P, _P, _u32, _P, _int]),
    "dsd_core_app": (_int, [_P, _int, _P, _P, _int, ctypes.POINTER(CoreAppResult)]),
    "dsd_batch_create": (_int, [_u32, _P, _P, _P, _P, _P, _int, _int, _P, ctypes.c_char_p,
                                ctypes.POINTER(_P)]),
    "dsd_batch_replay": (_int, [_P]),
    "dsd_set_checked": (_int, [_int]),
    "dsd_peel_app": (_int, [_P, _int, _P, _P, _int, ctypes.POINTER(PeelAppResult)]),
    "dsd_listing_bytes": (_int, [_P, _P, _P]),
    "dsd_checked_add_selftest": (_int, [_u64, _P, _u32, _P, _P]),
    "dsd_batch_run": (_int, [_int, _P, _P, _P, _P, ctypes.c_char_p]),
    "dsd_batch_results": (_int, [_P, _P, _P, _P]),
    "dsd_batch_info": (_int, [_P, _P, _P, _P, _P]),
    "dsd_batch_set_shape": (_int, [_P, _u32, _u32, _u32]),
    "dsd_batch_destroy": (None, [_P]),
    "dsd_triangle_degrees_noalloc": (_int, [_u32, _P, _P, _P, _P, _P]),
    "dsd_set_profiling": (_int, [_P, _int]),
    "dsd_phase_stats": (_int, [_P, _P, _P, _P]),
    "dsd_peel_stats": (_int, [_P, _int, _P]),
    "dsd_check_barrier_timeout": (_int, [_int, _u32, _P]),
    "dsd_model_param_count": (_u64, []),
    "dsd_model_create": (_int, [_u64, _P, ctypes.POINTER(_P)]),
    "dsd_model_destroy": (None, [_P]),
    "dsd_model_get_state": (_int, [_P, _P, _u64]),
    "dsd_model_set_state": (_int, [_P, _P, _u64]),
    "dsd_model_forward": (_int, [_P, _P, _u32, _P]),
    "dsd_model_gradient": (_int, [_P, _P, _P, _u32, ctypes.c_float, _P, _P]),
    "dsd_model_train_step": (_int, [_P, _P, _P, _u32, ctypes.c_float, ctypes.c_float, _P]),
    "dsd_graph_features": (_int, [_P, _int, _P, _int]),
    "dsd_core_app_seeded": (_int, [_P, _int, _P, _P, _P, _int, ctypes.POINTER(CoreAppResult)]),
    "dsd_core_app_seeded_info": (_int, [_P, _int, _P, _P, _P, _int, ctypes.POINTER(CoreAppResult),
                                   ctypes.POINTER(SeedInfo)]),
    "dsd_core_app_topdown": (_int, [_P, _int, _P, _P, _int, ctypes.POINTER(CoreAppResult),
                                    ctypes.POINTER(TopdownInfo)]),
    "dsd_core_exact": (_int, [_P, _int, _P, _int, ctypes.POINTER(ExactInfo)]),
    "dsd_pattern_degrees": (_int, [_P, _int, _int, _P, _P, _int]),
    "dsd_pattern_core_decompose": (_int, [_P, _int, _int, _P, _P, _P, _P, _P, _u32, _P, _int]),
    "dsd_pattern_core_app": (_int, [_P, _int, _int, _P, _P, _int,
                                    ctypes.POINTER(CoreAppResult)]),
}

PEEL_STATS = ("rounds", "levels", "items", "bytes", "barrier_ns", "barriers", "compactions",
              "threads", "grid", "kmax", "small_round",
              "t_large_retire", "t_large_scan", "t_large_jump", "t_large_enum",
              "t_small_retire", "t_small_jump", "t_small_mark", "t_small_enum",
              "tail_n", "tail_round", "tail_ns",
              "t_tail_build", "t_tail_front", "t_tail_jump", "t_tail_prefix", "t_tail_work",
              "t_tail_sync", "t_tail_retire")


def load(path: str = LIB_PATH):
    """Load libdsd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libdsd.so is not built (run __graft_entry__.build()); "
                           "there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        lib = load()
        raise DSDError(rc, (lib.dsd_last_error() or b"").decode())


# ----------------------------------------------------- raw C entry points

def dsd_status_string(s):
    return load().dsd_status_string(s).decode()


def dsd_last_error():
    return load().dsd_last_error().decode()


def dsd_version():
    return load().dsd_version().decode()


def dsd_kernel_launches():
    return int(load().dsd_kernel_launches())


def dsd_set_wait_limit_ms(ms):
    _check(load().dsd_set_wait_limit_ms(ms))


def dsd_listing_bytes(g):
    a = _u64()
    b = _u64()
    _check(load().dsd_listing_bytes(g, ctypes.addressof(a), ctypes.addressof(b)))
    return int(a.value), int(b.value)


def dsd_peel_app(g, h, densest_ptr, order_ptr, mem):
    r = PeelAppResult()
    _check(load().dsd_peel_app(g, h, densest_ptr, order_ptr, mem, ctypes.byref(r)))
    return r


def dsd_set_checked(on):
    _check(load().dsd_set_checked(1 if on else 0))


def dsd_checked_add_selftest(start, addends):
    a = np.ascontiguousarray(np.asarray(addends, np.uint64))
    out = _u64()
    flag = ctypes.c_int()
    _check(load().dsd_checked_add_selftest(int(start), _np_ptr(a) if a.size else 0, a.size,
                                           ctypes.addressof(out), ctypes.addressof(flag)))
    return int(out.value), bool(flag.value)


def dsd_set_peel_small_limit(max_alive):
    _check(load().dsd_set_peel_small_limit(max_alive))


def dsd_set_peel_tail_limit(max_alive):
    _check(load().dsd_set_peel_tail_limit(max_alive))


def dsd_set_peel_app_queue(shared_words, global_words):
    _check(load().dsd_set_peel_app_queue(shared_words, global_words))


def dsd_set_peel_items(warp_max, mid_max):
    _check(load().dsd_set_peel_items(warp_max, mid_max))


def dsd_graph_from_edges(n, m, src_ptr, dst_ptr, mem, stream_ptr):
    out = _P()
    _check(load().dsd_graph_from_edges(n, m, src_ptr, dst_ptr, mem, stream_ptr, ctypes.byref(out)))
    return out.value


def dsd_graph_from_csr(n, off_ptr, adj_ptr, mem, stream_ptr):
    out = _P()
    _check(load().dsd_graph_from_csr(n, off_ptr, adj_ptr, mem, stream_ptr, ctypes.byref(out)))
    return out.value


def dsd_graph_destroy(g):
    load().dsd_graph_destroy(g)


def dsd_graph_info(g):
    n = _u32()
    m = _u64()
    _check(load().dsd_graph_info(g, ctypes.addressof(n), ctypes.addressof(m)))
    return n.value, m.value


def dsd_graph_set_stream(g, stream_ptr):
    _check(load().dsd_graph_set_stream(g, stream_ptr))


def dsd_graph_csr(g, off_ptr, adj_ptr, mem):
    _check(load().dsd_graph_csr(g, off_ptr, adj_ptr, mem))


def dsd_degeneracy_order(g, core2_ptr, rank_ptr, degen_ptr, mem):
    _check(load().dsd_degeneracy_order(g, core2_ptr, rank_ptr, degen_ptr, mem))


def dsd_clique_degrees(g, h, deg_ptr, mu_ptr, mem):
    _check(load().dsd_clique_degrees(g, h, deg_ptr, mu_ptr, mem))


def dsd_core_decompose(g, h, core_ptr, kmax_ptr, mem):
    _check(load().dsd_core_decompose(g, h, core_ptr, kmax_ptr, mem))


def dsd_level_stats(g, h, k_ptr, size_ptr, mu_ptr, cap, nlevels_ptr, mem):
    _check(load().dsd_level_stats(g, h, k_ptr, size_ptr, mu_ptr, cap, nlevels_ptr, mem))


def dsd_core_app(g, h, kcore_ptr, densest_ptr, mem):
    r = CoreAppResult()
    _check(load().dsd_core_app(g, h, kcore_ptr, densest_ptr, mem, ctypes.byref(r)))
    return r


def dsd_batch_create(count, n_ptr, h_ptr, m_ptr, src_ptr, dst_ptr, mem, want_cores, stream_ptr,
                     autotune_cache=None):
    out = _P()
    cache = autotune_cache.encode() if autotune_cache else None
    _check(load().dsd_batch_create(count, n_ptr, h_ptr, m_ptr, src_ptr, dst_ptr, mem, want_cores,
                                   stream_ptr, cache, ctypes.byref(out)))
    return out.value


def dsd_batch_replay(b):
    _check(load().dsd_batch_replay(b))


def dsd_batch_run(graphs, hs, want_cores=False, autotune_cache=None):
    """CoreApp results (and core numbers when want_cores) for a list of
    graph handles (ints or Graph objects) with clique sizes hs."""
    count = len(graphs)
    hv = (ctypes.c_int * max(count, 1))(*[int(h) for h in hs])
    gv = (ctypes.c_void_p * max(count, 1))(*[int(getattr(g, "handle", g)) for g in graphs])
    res = (CoreAppResult * max(count, 1))()
    cores = None
    cptr = 0
    if want_cores:
        ns = [dsd_graph_info(int(getattr(g, "handle", g)))[0] for g in graphs]
        cores = [np.zeros(max(n, 1), np.uint64) for n in ns]
        cp = (ctypes.c_void_p * max(count, 1))(*[c.ctypes.data for c in cores])
        cptr = ctypes.addressof(cp)
    cache = autotune_cache.encode() if autotune_cache else None
    _check(load().dsd_batch_run(count, ctypes.addressof(gv), ctypes.addressof(hv),
                                ctypes.addressof(res), cptr, cache))
    out = []
    for i in range(count):
        r = res[i]
        d = dict(kmax=int(r.kmax), kmax_core_size=int(r.kmax_core_size),
                 kmax_core_mu=int(r.kmax_core_mu), best_k=int(r.best_k),
                 densest_size=int(r.densest_size), densest_mu=int(r.densest_mu),
                 nlevels=int(r.nlevels))
        if cores is not None:
            d["core"] = cores[i][: ns[i]]
        out.append(d)
    return out


def dsd_batch_results(b, res_ptr, status_ptr, cores_ptr):
    _check(load().dsd_batch_results(b, res_ptr, status_ptr, cores_ptr))


def dsd_batch_info(b):
    t = _u32()
    c = _u32()
    lp = _u32()
    ms = ctypes.c_float()
    _check(load().dsd_batch_info(b, ctypes.addressof(t), ctypes.addressof(c),
                                 ctypes.addressof(lp), ctypes.addressof(ms)))
    return t.value, c.value, lp.value, ms.value


def dsd_batch_set_shape(b, threads, ctas_per_sm, lanes_per_row):
    _check(load().dsd_batch_set_shape(b, threads, ctas_per_sm, lanes_per_row))


def dsd_batch_destroy(b):
    load().dsd_batch_destroy(b)


class Batch:
    """Many small graphs run by one persistent launch (captured in a CUDA
    graph).  graphs: list of (n, src, dst, h) with numpy edge arrays."""

    def __init__(self, graphs, want_cores=True, stream=None, autotune_cache=None):
        self.count = len(graphs)
        self.n = np.array([g[0] for g in graphs], np.uint32)
        self.h = np.array([g[3] for g in graphs], np.int32)
        self.m = np.array([len(g[1]) for g in graphs], np.uint64)
        src = np.concatenate([np.asarray(g[1], np.uint32) for g in graphs]) if graphs else np.zeros(0, np.uint32)
        dst = np.concatenate([np.asarray(g[2], np.uint32) for g in graphs]) if graphs else np.zeros(0, np.uint32)
        self.src = np.ascontiguousarray(src)
        self.dst = np.ascontiguousarray(dst)
        self.want_cores = bool(want_cores)
        sp = _stream_ptr(stream)
        self.handle = dsd_batch_create(self.count, _np_ptr(self.n), _np_ptr(self.h), _np_ptr(self.m),
                                       _np_ptr(self.src) if self.src.size else 0,
                                       _np_ptr(self.dst) if self.dst.size else 0, DSD_MEM_HOST,
                                       1 if want_cores else 0, sp, autotune_cache)

    def run(self):
        dsd_batch_replay(self.handle)

    def results(self):
        res = (CoreAppResult * max(self.count, 1))()
        status = np.zeros(max(self.count, 1), np.int32)
        cores = np.zeros(max(int(self.n.sum()), 1), np.uint64) if self.want_cores else None
        dsd_batch_results(self.handle, ctypes.addressof(res), _np_ptr(status),
                          _np_ptr(cores) if cores is not None else 0)
        out = []
        pos = 0
        for i in range(self.count):
            r = res[i]
            d = dict(kmax=int(r.kmax), kmax_core_size=int(r.kmax_core_size),
                     kmax_core_mu=int(r.kmax_core_mu), best_k=int(r.best_k),
                     densest_size=int(r.densest_size), densest_mu=int(r.densest_mu),
                     nlevels=int(r.nlevels), status=int(status[i]))
            if cores is not None:
                d["core"] = cores[pos:pos + int(self.n[i])]
            pos += int(self.n[i])
            out.append(d)
        return out

    def info(self):
        """(threads, ctas_per_sm, lanes_per_row, tuned_ms)"""
        return dsd_batch_info(self.handle)

    def set_shape(self, threads, ctas_per_sm, lanes_per_row):
        dsd_batch_set_shape(self.handle, threads, ctas_per_sm, lanes_per_row)

    def close(self):
        if self.handle:
            dsd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dsd_triangle_degrees_noalloc(n, off_ptr, adj_ptr, deg_ptr, mu_ptr, stream_ptr):
    _check(load().dsd_triangle_degrees_noalloc(n, off_ptr, adj_ptr, deg_ptr, mu_ptr, stream_ptr))


def dsd_set_profiling(g, on):
    _check(load().dsd_set_profiling(g, 1 if on else 0))


def dsd_phase_stats(g):
    ms = (ctypes.c_float * DSD_NPHASES)()
    by = (ctypes.c_uint64 * DSD_NPHASES)()
    la = (ctypes.c_uint32 * DSD_NPHASES)()
    _check(load().dsd_phase_stats(g, ctypes.addressof(ms), ctypes.addressof(by),
                                  ctypes.addressof(la)))
    return list(ms), list(by), list(la)


def dsd_peel_stats(g, which):
    out = (ctypes.c_uint64 * len(PEEL_STATS))()
    _check(load().dsd_peel_stats(g, which, ctypes.addressof(out)))
    return dict(zip(PEEL_STATS, [int(x) for x in out]))


def dsd_check_barrier_timeout(absent_block, wait_ms, stream_ptr):
    _check(load().dsd_check_barrier_timeout(absent_block, wait_ms, stream_ptr))


def dsd_model_param_count():
    return int(load().dsd_model_param_count())


def dsd_model_create(seed, stream_ptr):
    out = _P()
    _check(load().dsd_model_create(seed, stream_ptr, ctypes.byref(out)))
    return out.value


def dsd_model_destroy(m):
    load().dsd_model_destroy(m)


def dsd_model_get_state(m, state_ptr, count):
    _check(load().dsd_model_get_state(m, state_ptr, count))


def dsd_model_set_state(m, state_ptr, count):
    _check(load().dsd_model_set_state(m, state_ptr, count))


def dsd_model_forward(m, x_ptr, B, out_ptr):
    _check(load().dsd_model_forward(m, x_ptr, B, out_ptr))


def dsd_model_gradient(m, x_ptr, y_ptr, B, q, loss_ptr, grad_ptr):
    _check(load().dsd_model_gradient(m, x_ptr, y_ptr, B, q, loss_ptr, grad_ptr))


def dsd_model_train_step(m, x_ptr, y_ptr, B, q, lr, loss_ptr):
    _check(load().dsd_model_train_step(m, x_ptr, y_ptr, B, q, lr, loss_ptr))


def dsd_graph_features(g, h, f_ptr, mem):
    _check(load().dsd_graph_features(g, h, f_ptr, mem))


def dsd_core_app_seeded(g, h, model, kcore_ptr, densest_ptr, mem):
    r = CoreAppResult()
    _check(load().dsd_core_app_seeded(g, h, model, kcore_ptr, densest_ptr, mem, ctypes.byref(r)))
    return r


def dsd_core_app_seeded_info(g, h, model, kcore_ptr, densest_ptr, mem):
    r = CoreAppResult()
    info = SeedInfo()
    _check(load().dsd_core_app_seeded_info(g, h, model, kcore_ptr, densest_ptr, mem,
                                           ctypes.byref(r), ctypes.byref(info)))
    return r, info


def dsd_pattern_degrees(g, pattern, x, deg_ptr, mu_ptr, mem):
    _check(load().dsd_pattern_degrees(g, pattern, x, deg_ptr, mu_ptr, mem))


def dsd_pattern_core_decompose(g, pattern, x, core_ptr, kmax_ptr, lk_ptr, ls_ptr, lm_ptr, cap,
                               nl_ptr, mem):
    _check(load().dsd_pattern_core_decompose(g, pattern, x, core_ptr, kmax_ptr, lk_ptr, ls_ptr,
                                             lm_ptr, cap, nl_ptr, mem))


def dsd_pattern_core_app(g, pattern, x, kcore_ptr, densest_ptr, mem):
    r = CoreAppResult()
    _check(load().dsd_pattern_core_app(g, pattern, x, kcore_ptr, densest_ptr, mem,
                                       ctypes.byref(r)))
    return r


def dsd_core_exact(g, h, cds_ptr, mem):
    info = ExactInfo()
    _check(load().dsd_core_exact(g, h, cds_ptr, mem, ctypes.byref(info)))
    return info


def dsd_core_app_topdown(g, h, kcore_ptr, densest_ptr, mem):
    r = CoreAppResult()
    info = TopdownInfo()
    _check(load().dsd_core_app_topdown(g, h, kcore_ptr, densest_ptr, mem, ctypes.byref(r),
                                       ctypes.byref(info)))
    return r, info


class Model:
    """Owns one dsd_model handle (the density-proposal network).  Inputs and
    outputs are float32 numpy arrays; the arithmetic runs in libdsd."""

    def __init__(self, seed=0, stream=None):
        self.stream_ptr = _stream_ptr(stream)
        self.handle = dsd_model_create(seed, self.stream_ptr)
        self.count = dsd_model_param_count()

    def close(self):
        if self.handle:
            dsd_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def state(self):
        st = np.zeros(3 * self.count + 1, np.float32)
        dsd_model_get_state(self.handle, _np_ptr(st), self.count)
        return st

    def set_state(self, st):
        st = np.ascontiguousarray(st, np.float32)
        if st.size != 3 * self.count + 1:
            raise ValueError("state has %d floats, expected %d" % (st.size, 3 * self.count + 1))
        dsd_model_set_state(self.handle, _np_ptr(st), self.count)

    @staticmethod
    def _x(X):
        X = np.ascontiguousarray(X, np.float32)
        if X.ndim != 2 or X.shape[1] != NFEAT:
            raise ValueError("features must be B x %d" % NFEAT)
        return X

    def forward(self, X):
        X = self._x(X)
        out = np.zeros(max(X.shape[0], 1), np.float32)
        dsd_model_forward(self.handle, _np_ptr(X), X.shape[0], _np_ptr(out))
        return out[: X.shape[0]]

    def gradient(self, X, y, q):
        X = self._x(X)
        y = np.ascontiguousarray(y, np.float32)
        loss = np.zeros(1, np.float32)
        grad = np.zeros(self.count, np.float32)
        dsd_model_gradient(self.handle, _np_ptr(X), _np_ptr(y), X.shape[0], q, _np_ptr(loss),
                           _np_ptr(grad))
        return float(loss[0]), grad

    def train_step(self, X, y, q, lr):
        X = self._x(X)
        y = np.ascontiguousarray(y, np.float32)
        loss = np.zeros(1, np.float32)
        dsd_model_train_step(self.handle, _np_ptr(X), _np_ptr(y), X.shape[0], q, lr,
                             _np_ptr(loss))
        return float(loss[0])


# -------------------------------------------------------- convenience

def _np_ptr(a):
    return a.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Graph:
    """Owns one dsd_graph handle.  ``mem`` selects host (numpy) or device
    (torch CUDA tensors) outputs for the query methods."""

    def __init__(self, handle, stream_ptr, keepalive=()):
        self.handle = handle
        self.stream_ptr = stream_ptr
        self._keep = keepalive
        self.n, self.m = dsd_graph_info(handle)

    # construction -----------------------------------------------------
    @classmethod
    def from_edges(cls, n, src, dst, stream=None):
        sp = _stream_ptr(stream)
        if hasattr(src, "is_cuda") and src.is_cuda:
            src = src.contiguous()
            dst = dst.contiguous()
            h = dsd_graph_from_edges(n, src.numel(), src.data_ptr(), dst.data_ptr(),
                                     DSD_MEM_DEVICE, sp)
        else:
            src = np.ascontiguousarray(src, np.uint32)
            dst = np.ascontiguousarray(dst, np.uint32)
            h = dsd_graph_from_edges(n, src.size, _np_ptr(src), _np_ptr(dst), DSD_MEM_HOST, sp)
        return cls(h, sp)

    @classmethod
    def from_csr(cls, n, off, adj, stream=None):
        sp = _stream_ptr(stream)
        if hasattr(off, "is_cuda") and off.is_cuda:
            h = dsd_graph_from_csr(n, off.data_ptr(), adj.data_ptr(), DSD_MEM_DEVICE, sp)
        else:
            off = np.ascontiguousarray(off, np.uint64)
            adj = np.ascontiguousarray(adj, np.uint32)
            h = dsd_graph_from_csr(n, _np_ptr(off), _np_ptr(adj) if adj.size else 0,
                                   DSD_MEM_HOST, sp)
        return cls(h, sp)

    def close(self):
        if self.handle:
            dsd_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # buffers ------------------------------------------------------------
    @staticmethod
    def _alloc(count, kind, mem):
        if mem == "host":
            return np.zeros(max(count, 1), np.uint64 if kind == 8 else np.uint32)
        import torch
        return torch.zeros(max(count, 1), dtype=torch.int64 if kind == 8 else torch.int32,
                           device="cuda")

    @staticmethod
    def _ptr(buf):
        return _np_ptr(buf) if isinstance(buf, np.ndarray) else buf.data_ptr()

    @staticmethod
    def _memc(mem):
        return DSD_MEM_HOST if mem == "host" else DSD_MEM_DEVICE

    # queries --------------------------------------------------------------
    def csr(self, mem="host"):
        off = self._alloc(self.n + 1, 8, mem)
        adj = self._alloc(2 * self.m, 4, mem)
        dsd_graph_csr(self.handle, self._ptr(off), self._ptr(adj), self._memc(mem))
        return off[: self.n + 1], adj[: 2 * self.m]

    def degeneracy_order(self, mem="host"):
        core2 = self._alloc(self.n, 4, mem)
        rank = self._alloc(self.n, 4, mem)
        dg = np.zeros(1, np.uint32)
        dsd_degeneracy_order(self.handle, self._ptr(core2), self._ptr(rank), _np_ptr(dg),
                             DSD_MEM_HOST if mem == "host" else DSD_MEM_DEVICE) \
            if mem == "host" else \
            dsd_degeneracy_order(self.handle, self._ptr(core2), self._ptr(rank), 0, DSD_MEM_DEVICE)
        return core2[: self.n], rank[: self.n], int(dg[0])

    def clique_degrees(self, h, mem="host"):
        deg = self._alloc(self.n, 8, mem)
        mu = self._alloc(1, 8, mem)
        dsd_clique_degrees(self.handle, h, self._ptr(deg), self._ptr(mu), self._memc(mem))
        return deg[: self.n], int(mu[0])

    def core_decompose(self, h, mem="host"):
        core = self._alloc(self.n, 8, mem)
        km = np.zeros(1, np.uint64)
        dsd_core_decompose(self.handle, h, self._ptr(core), _np_ptr(km), DSD_MEM_HOST) \
            if mem == "host" else None
        if mem != "host":
            kmd = self._alloc(1, 8, mem)
            dsd_core_decompose(self.handle, h, self._ptr(core), self._ptr(kmd), DSD_MEM_DEVICE)
            km[0] = int(kmd[0])
        return core[: self.n], int(km[0])

    def level_stats(self, h):
        nl = np.zeros(1, np.uint32)
        cap = self.n + 1
        k = np.zeros(cap, np.uint64)
        s = np.zeros(cap, np.uint32)
        mu = np.zeros(cap, np.uint64)
        dsd_level_stats(self.handle, h, _np_ptr(k), _np_ptr(s), _np_ptr(mu), cap, _np_ptr(nl),
                        DSD_MEM_HOST)
        c = int(nl[0])
        return k[:c], s[:c], mu[:c]

    def peel_app(self, h, mem="host"):
        """PeelApp (Algorithm 2): the set, its mu and size, the removal order."""
        de = self._alloc(self.n, 4, mem)
        od = self._alloc(self.n, 4, mem)
        r = dsd_peel_app(self.handle, h, self._ptr(de), self._ptr(od), self._memc(mem))
        return dict(set=de[: r.size], mu=int(r.mu), size=int(r.size), removed=int(r.removed),
                    level_k=int(r.level_k), order=od[: self.n])

    def core_app(self, h, mem="host", sets=True):
        kc = self._alloc(self.n, 4, mem) if sets else None
        de = self._alloc(self.n, 4, mem) if sets else None
        r = dsd_core_app(self.handle, h, self._ptr(kc) if sets else 0,
                         self._ptr(de) if sets else 0, self._memc(mem))
        out = dict(kmax=int(r.kmax), kmax_core_mu=int(r.kmax_core_mu), best_k=int(r.best_k),
                   densest_mu=int(r.densest_mu), densest_size=int(r.densest_size),
                   kmax_core_size=int(r.kmax_core_size), nlevels=int(r.nlevels))
        if sets:
            out["kmax_core"] = kc[: r.kmax_core_size]
            out["densest"] = de[: r.densest_size]
        return out

    def features(self, h):
        f = np.zeros(NFEAT, np.float32)
        dsd_graph_features(self.handle, h, _np_ptr(f), DSD_MEM_HOST)
        return f

    def core_app_seeded(self, h, model, mem="host", sets=True):
        kc = self._alloc(self.n, 4, mem) if sets else None
        de = self._alloc(self.n, 4, mem) if sets else None
        r, info = dsd_core_app_seeded_info(self.handle, h, model.handle,
                                           self._ptr(kc) if sets else 0,
                                           self._ptr(de) if sets else 0, self._memc(mem))
        out = dict(kmax=int(r.kmax), kmax_core_mu=int(r.kmax_core_mu), best_k=int(r.best_k),
                   densest_mu=int(r.densest_mu), densest_size=int(r.densest_size),
                   kmax_core_size=int(r.kmax_core_size), nlevels=int(r.nlevels),
                   seeded_accepted=int(r.seeded_accepted), seed_k=int(r.seed_k))
        if sets:
            out["kmax_core"] = kc[: r.kmax_core_size]
            out["densest"] = de[: r.densest_size]
        out["seed"] = dict(rho_prime=float(info.rho_prime), accepted=int(info.accepted),
                           seed_k=int(info.seed_k), x0=int(info.x0), sub_n=int(info.sub_n),
                           sub_m=int(info.sub_m))
        return out

    def core_app_topdown(self, h, mem="host", sets=True):
        kc = self._alloc(self.n, 4, mem) if sets else None
        de = self._alloc(self.n, 4, mem) if sets else None
        r, info = dsd_core_app_topdown(self.handle, h, self._ptr(kc) if sets else 0,
                                       self._ptr(de) if sets else 0, self._memc(mem))
        out = dict(kmax=int(r.kmax), kmax_core_mu=int(r.kmax_core_mu), best_k=int(r.best_k),
                   densest_mu=int(r.densest_mu), densest_size=int(r.densest_size),
                   kmax_core_size=int(r.kmax_core_size), nlevels=int(r.nlevels))
        if sets:
            out["kmax_core"] = kc[: r.kmax_core_size]
            out["densest"] = de[: r.densest_size]
        out["schedule"] = dict(passes=int(info.passes), sub_n=int(info.sub_n), x=int(info.x),
                               gamma_out=int(info.gamma_out), sub_m=int(info.sub_m))
        return out

    # patterns (Sec. 6) -----------------------------------------------------
    def pattern_degrees(self, pattern, x=0, mem="host"):
        deg = self._alloc(self.n, 8, mem)
        mu = self._alloc(1, 8, mem)
        dsd_pattern_degrees(self.handle, pattern, x, self._ptr(deg), self._ptr(mu),
                            self._memc(mem))
        return deg[: self.n], int(mu[0])

    def pattern_core_decompose(self, pattern, x=0):
        """(core numbers, k_max, level k, |R_k|, mu(R_k)) for a pattern."""
        core = np.zeros(max(self.n, 1), np.uint64)
        km = np.zeros(1, np.uint64)
        nl = np.zeros(1, np.uint32)
        cap = max(self.n, 1)
        lk = np.zeros(cap, np.uint64)
        ls = np.zeros(cap, np.uint32)
        lm = np.zeros(cap, np.uint64)
        dsd_pattern_core_decompose(self.handle, pattern, x, _np_ptr(core), _np_ptr(km),
                                   _np_ptr(lk), _np_ptr(ls), _np_ptr(lm), cap, _np_ptr(nl),
                                   DSD_MEM_HOST)
        k = int(nl[0])
        return core[: self.n], int(km[0]), lk[:k], ls[:k], lm[:k]

    def pattern_core_app(self, pattern, x=0, mem="host"):
        kc = self._alloc(self.n, 4, mem)
        de = self._alloc(self.n, 4, mem)
        r = dsd_pattern_core_app(self.handle, pattern, x, self._ptr(kc), self._ptr(de),
                                 self._memc(mem))
        return dict(kmax=int(r.kmax), kmax_core=kc[: r.kmax_core_size],
                    kmax_core_mu=int(r.kmax_core_mu), best_k=int(r.best_k),
                    densest=de[: r.densest_size], densest_mu=int(r.densest_mu),
                    densest_size=int(r.densest_size), nlevels=int(r.nlevels))

    def core_exact(self, h, mem="host", sets=True):
        """CoreExact: rho_opt = mu / size and the largest densest set."""
        cds = self._alloc(self.n, 4, mem) if sets else None
        info = dsd_core_exact(self.handle, h, self._ptr(cds) if sets else 0, self._memc(mem))
        out = {f: int(getattr(info, f)) for f, _ in ExactInfo._fields_ if f != "reserved"}
        if sets:
            out["cds"] = cds[: info.size]
        return out

    def set_profiling(self, on=True):
        dsd_set_profiling(self.handle, on)

    def phase_stats(self):
        ms, by, la = dsd_phase_stats(self.handle)
        return {p: dict(ms=ms[i], bytes=by[i], launches=la[i]) for i, p in enumerate(PHASES)}
