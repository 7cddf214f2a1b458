"""ctypes binding of libspider.so: argument marshalling only.

Every function mirrors one entry point of include/spider.h with the same name;
all computation happens in the library's CUDA kernels.  Importing this module
does not touch the GPU; the first call loads the library and raises if it is
missing (there is no fallback path)."""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libspider.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "spider.h")

SPIDER_OK = 0
ERRORS = {-1: "INVAL", -2: "OOM", -3: "CUDA", -4: "NONFINITE", -5: "TIMEOUT", -6: "UNSUPPORTED"}
TT_HOMOGENEOUS, TT_LINEAR_GRADIENT, TT_MLP = 0, 1, 2
FP32, BF16, FP8 = 0, 1, 2
UPDATE_SGLD, UPDATE_PSGLD, UPDATE_ADAM = 0, 1, 2
LOSS_WHITENED, LOSS_L1 = 0, 1


class SpiderError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"spider error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class spider_catalog(C.Structure):
    _fields_ = [("M", C.c_int64), ("N", C.c_int64), ("xyzt0", C.POINTER(C.c_double)),
                ("i", C.POINTER(C.c_int32)), ("j", C.POINTER(C.c_int32)), ("k", C.POINTER(C.c_int32)),
                ("dt", C.POINTER(C.c_double)), ("w", C.POINTER(C.c_float))]


class spider_stations(C.Structure):
    _fields_ = [("S", C.c_int32), ("xyz", C.POINTER(C.c_double))]


class spider_net(C.Structure):
    _fields_ = [("kind", C.c_int32), ("v0", C.c_double), ("g", C.c_double), ("H", C.c_int32),
                ("W", C.POINTER(C.c_float) * 5), ("b", C.POINTER(C.c_float) * 5)]


class spider_config(C.Structure):
    _fields_ = [("sigma", C.c_double), ("kappa", C.c_double), ("p", C.c_double), ("ell", C.c_double),
                ("eps_w", C.c_double), ("sig_e", C.c_double * 4), ("sig_c", C.c_double * 4),
                ("batch_n", C.c_int64), ("block_obs", C.c_int64), ("precision", C.c_int32),
                ("thin", C.c_int32), ("reorder", C.c_int32), ("chain", C.c_int32),
                ("catalog", C.c_int32), ("noise_scale", C.c_float), ("pcg_max_it", C.c_int32),
                ("pcg_tol", C.c_float), ("sample_cap", C.c_int64), ("update", C.c_int32),
                ("beta1", C.c_float), ("beta2", C.c_float), ("upd_eps", C.c_float), ("loss", C.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libspider.so (raises FileNotFoundError if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: run __graft_entry__.build() first")
    L = C.CDLL(path)
    vp, i64, i32, u64, u32, f32 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_uint32, C.c_float
    pd, pf, pi64 = C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_int64)
    sig = {
        "spider_config_default": (None, [C.POINTER(spider_config)]),
        "spider_create": (C.c_int, [C.POINTER(spider_catalog), C.POINTER(spider_stations),
                                    C.POINTER(spider_net), C.POINTER(spider_config), vp, C.POINTER(vp)]),
        "spider_create_batch": (C.c_int, [i32, C.POINTER(spider_catalog), C.POINTER(spider_stations),
                                          C.POINTER(spider_net), C.POINTER(spider_config), i32, vp,
                                          C.POINTER(vp)]),
        "spider_grad_logpost": (C.c_int, [vp, u64, pf, pd]),
        "spider_sgld_step": (C.c_int, [vp, f32, u64]),
        "spider_samples": (C.c_int, [vp, pd, i64, pi64]),
        "spider_get_state": (C.c_int, [vp, pd, pi64]),
        "spider_set_state": (C.c_int, [vp, pd, i64]),
        "spider_get_moments": (C.c_int, [vp, pd, pd]),
        "spider_set_noise_scale": (C.c_int, [vp, f32]),
        "spider_set_moments": (C.c_int, [vp, pd, pd]),
        "spider_outlier_mask": (C.c_int, [vp, C.c_double, C.POINTER(C.c_uint8), pi64, pd, pd]),
        "spider_linearisation_mask": (C.c_int, [vp, C.c_double, C.POINTER(C.c_uint8), pi64]),
        "spider_uq": (C.c_int, [vp, pd, C.c_double, C.c_double, pd, pd, pd, pd]),
        "spider_sync": (C.c_int, [vp]),
        "spider_set_timing": (C.c_int, [vp, C.c_int]),
        "spider_set_wait_limit_ns": (C.c_int, [vp, u64]),
        "spider_last_kernel_timing": (C.c_int, [vp, pf, pi64]),
        "spider_last_whiten_timing": (C.c_int, [vp, pf]),
        "spider_last_timing": (C.c_int, [vp, pf, pi64, pi64, C.POINTER(i32)]),
        "spider_debug_blocks": (C.c_int, [vp, pi64, i64, pi64]),
        "spider_debug_obs": (C.c_int, [vp, pi64, pf, pf, i64, pi64]),
        "spider_last_error": (C.c_char_p, [vp]),
        "spider_info": (C.c_int, [vp, pi64, i32]),
        "spider_set_tuning": (C.c_int, [vp, C.POINTER(i32), i32]),
        "spider_diagnostics": (C.c_int, [vp, u64, f32, pd, pd]),
        "spider_destroy": (None, [vp]),
        "spider_net_upload": (C.c_int, [C.POINTER(spider_net), i32, C.POINTER(vp)]),
        "spider_net_free": (None, [vp]),
        "spider_tt_pairs": (C.c_int, [vp, i64, vp, vp, vp, vp, vp, vp]),
        "spider_philox_words": (C.c_int, [u64, u32, u32, u32, u32, i64, C.POINTER(u32)]),
        "spider_tt_pairs_noalloc": (C.c_int, [C.POINTER(spider_net), i64, vp, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def declared_symbols(header: str = HEADER):
    """Names of the functions include/spider.h declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(spider_[a-z0-9_]+)\s*\(", text))
    # "int spider_get_state/ spider_set_state" style lines are not used; keep function names only
    return sorted(n for n in names if not n.startswith("spider_catalog"))


def _check(code, ctx=None):
    if code != SPIDER_OK:
        msg = load_library().spider_last_error(ctx)
        raise SpiderError(code, msg.decode() if msg else "")


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def config_default() -> spider_config:
    c = spider_config()
    load_library().spider_config_default(C.byref(c))
    return c


def make_config(**kw) -> spider_config:
    c = config_default()
    for key, val in kw.items():
        if key in ("sig_e", "sig_c"):
            arr = getattr(c, key)
            for a in range(4):
                arr[a] = float(val[a])
        else:
            setattr(c, key, val)
    return c


class Net:
    """Host-side description of a travel-time model (keeps its arrays alive)."""

    def __init__(self, kind: int, v0: float = 0.0, g: float = 0.0, mlp: Optional[dict] = None):
        self.s = spider_net()
        self.s.kind = kind
        self.s.v0 = v0
        self.s.g = g
        self._keep = []
        if mlp is not None:
            self.s.H = int(mlp["H"])
            for l in range(5):
                W = np.ascontiguousarray(mlp["W"][l], dtype=np.float32)
                b = np.ascontiguousarray(mlp["b"][l], dtype=np.float32)
                self._keep += [W, b]
                self.s.W[l] = _ptr(W, C.c_float)
                self.s.b[l] = _ptr(b, C.c_float)


def net_for_catalog(cat) -> Net:
    if cat.spec.forward == "mlp":
        return Net(TT_MLP, mlp=cat.net)
    return Net(TT_HOMOGENEOUS, v0=6.0)


def config_for_catalog(cat, **over) -> spider_config:
    h = cat.spec.hyper
    kw = dict(sigma=h.sigma, kappa=h.kappa, p=h.p, ell=h.ell, eps_w=h.eps_w, sig_e=h.sig_e,
              sig_c=h.sig_c, batch_n=h.batch_n, block_obs=h.block_obs)
    kw.update(over)
    return make_config(**kw)


class Context:
    """Owns a spider_ctx (spider_create ... spider_destroy)."""

    def __init__(self, xyzt0, i, j, k, dt, stations, net: Net, cfg: spider_config,
                 w=None, stream: Optional[int] = None):
        L = load_library()
        self._arrays = dict(
            xyzt0=np.ascontiguousarray(xyzt0, dtype=np.float64),
            i=np.ascontiguousarray(i, dtype=np.int32), j=np.ascontiguousarray(j, dtype=np.int32),
            k=np.ascontiguousarray(k, dtype=np.int32), dt=np.ascontiguousarray(dt, dtype=np.float64),
            sta=np.ascontiguousarray(stations, dtype=np.float64))
        a = self._arrays
        self.M, self.N = a["xyzt0"].shape[0], a["i"].shape[0]
        self.n_sub = 1
        cat = spider_catalog(self.M, self.N, _ptr(a["xyzt0"], C.c_double), _ptr(a["i"], C.c_int32),
                             _ptr(a["j"], C.c_int32), _ptr(a["k"], C.c_int32),
                             _ptr(a["dt"], C.c_double), None)
        if w is not None:
            a["w"] = np.ascontiguousarray(w, dtype=np.float32)
            cat.w = _ptr(a["w"], C.c_float)
        sta = spider_stations(a["sta"].shape[0], _ptr(a["sta"], C.c_double))
        self.net = net
        self.cfg = cfg
        h = C.c_void_p()
        code = L.spider_create(C.byref(cat), C.byref(sta), C.byref(net.s), C.byref(cfg),
                               C.c_void_p(stream) if stream else None, C.byref(h))
        _check(code, None)
        self.h = h
        # the library copied everything it keeps
        self._arrays = None

    @classmethod
    def batch(cls, cats, chains: int, net: Net, cfg: spider_config, stream: Optional[int] = None):
        """spider_create_batch over synthetic catalogs (list), `chains` chains each."""
        self = cls.__new__(cls)
        L = load_library()
        keep = []
        ccats = (spider_catalog * len(cats))()
        cstas = (spider_stations * len(cats))()
        for a, cat in enumerate(cats):
            arr = [np.ascontiguousarray(cat.init_xyzt, dtype=np.float64),
                   np.ascontiguousarray(cat.i, dtype=np.int32), np.ascontiguousarray(cat.j, dtype=np.int32),
                   np.ascontiguousarray(cat.k, dtype=np.int32), np.ascontiguousarray(cat.dt, dtype=np.float64),
                   np.ascontiguousarray(cat.stations, dtype=np.float64)]
            keep += arr
            ccats[a] = spider_catalog(cat.M, cat.N, _ptr(arr[0], C.c_double), _ptr(arr[1], C.c_int32),
                                      _ptr(arr[2], C.c_int32), _ptr(arr[3], C.c_int32),
                                      _ptr(arr[4], C.c_double), None)
            cstas[a] = spider_stations(cat.S, _ptr(arr[5], C.c_double))
        h = C.c_void_p()
        _check(L.spider_create_batch(len(cats), ccats, cstas, C.byref(net.s), C.byref(cfg), chains,
                                     C.c_void_p(stream) if stream else None, C.byref(h)), None)
        self.h = h
        self.net = net
        self.cfg = cfg
        self.M = sum(c.M for c in cats) * chains
        self.N = sum(c.N for c in cats) * chains
        self.n_sub = len(cats) * chains
        self._arrays = None
        return self

    @classmethod
    def from_catalog(cls, cat, net: Optional[Net] = None, **cfg_over):
        cfg = config_for_catalog(cat, **cfg_over)
        return cls(cat.init_xyzt, cat.i, cat.j, cat.k, cat.dt, cat.stations,
                   net or net_for_catalog(cat), cfg)

    def close(self):
        if getattr(self, "h", None):
            load_library().spider_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- entry points
    def spider_grad_logpost(self, batch_seed: int = 0, want_grad: bool = True):
        g = np.empty((self.M, 4), np.float32) if want_grad else None
        lp = C.c_double()
        _check(load_library().spider_grad_logpost(self.h, C.c_uint64(batch_seed),
                                                  _ptr(g, C.c_float) if want_grad else None,
                                                  C.byref(lp)), self.h)
        return g, lp.value

    def spider_sgld_step(self, eps: float, batch_seed: int):
        _check(load_library().spider_sgld_step(self.h, C.c_float(eps), C.c_uint64(batch_seed)), self.h)

    def spider_samples(self, cap: int):
        out = np.empty((max(cap, 0), self.M, 4), np.float64)
        n = C.c_int64()
        _check(load_library().spider_samples(self.h, _ptr(out, C.c_double), cap, C.byref(n)), self.h)
        return out[: n.value]

    def spider_get_state(self, out_ptr: Optional[int] = None):
        """(theta M x 4 FP64 in the caller's order, step).  With out_ptr (the
        address of a host buffer of M x 4 doubles, e.g. page-locked memory) the
        state is written there and None is returned in place of the array."""
        st = C.c_int64()
        if out_ptr is not None:
            _check(load_library().spider_get_state(self.h, C.cast(C.c_void_p(out_ptr), C.POINTER(C.c_double)),
                                                   C.byref(st)), self.h)
            return None, st.value
        th = np.empty((self.M, 4), np.float64)
        _check(load_library().spider_get_state(self.h, _ptr(th, C.c_double), C.byref(st)), self.h)
        return th, st.value

    def spider_set_state(self, theta, step: int):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        _check(load_library().spider_set_state(self.h, _ptr(th, C.c_double), int(step)), self.h)

    def spider_set_noise_scale(self, scale: float):
        _check(load_library().spider_set_noise_scale(self.h, float(scale)), self.h)

    def spider_get_moments(self):
        """(m, v) moment states of the pSGLD / Adam updates, M x 4 each."""
        m = np.empty((self.M, 4), np.float64)
        v = np.empty((self.M, 4), np.float64)
        _check(load_library().spider_get_moments(self.h, _ptr(m, C.c_double), _ptr(v, C.c_double)), self.h)
        return m, v

    def spider_set_moments(self, m=None, v=None):
        mm = None if m is None else np.ascontiguousarray(m, dtype=np.float64)
        vv = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        _check(load_library().spider_set_moments(
            self.h, _ptr(mm, C.c_double) if mm is not None else None,
            _ptr(vv, C.c_double) if vv is not None else None), self.h)

    def spider_outlier_mask(self, k_mad: float = 4.0):
        """(keep mask over the caller's observations, median and MAD per sub-problem)."""
        keep = np.empty(self.N, np.uint8)
        kept = C.c_int64()
        ns = self.n_sub
        med = np.empty(ns, np.float64)
        mad = np.empty(ns, np.float64)
        _check(load_library().spider_outlier_mask(self.h, float(k_mad), _ptr(keep, C.c_uint8), C.byref(kept),
                                                  _ptr(med, C.c_double), _ptr(mad, C.c_double)), self.h)
        assert int(keep.sum()) == kept.value
        return keep.astype(bool), med, mad

    def spider_linearisation_mask(self, max_rel: float = 0.05):
        """Keep mask over the caller's observations (linearisation error <= max_rel)."""
        keep = np.empty(self.N, np.uint8)
        kept = C.c_int64()
        _check(load_library().spider_linearisation_mask(self.h, float(max_rel), _ptr(keep, C.c_uint8),
                                                        C.byref(kept)), self.h)
        assert int(keep.sum()) == kept.value
        return keep.astype(bool)

    def spider_uq(self, truth=None, lo_pct: float = 0.5, hi_pct: float = 99.5):
        """Per event and coordinate: median, credible half-width, calibration
        percentile of the truth (NaN without truth) and effective sample size."""
        out = [np.empty((self.M, 4), np.float64) for _ in range(4)]
        tr = None if truth is None else np.ascontiguousarray(truth, dtype=np.float64)
        _check(load_library().spider_uq(self.h, _ptr(tr, C.c_double) if tr is not None else None,
                                        float(lo_pct), float(hi_pct), *(_ptr(o, C.c_double) for o in out)),
               self.h)
        return dict(median=out[0], halfwidth=out[1], calib=out[2], ess=out[3])

    def spider_sync(self):
        _check(load_library().spider_sync(self.h), self.h)

    def spider_last_kernel_timing(self):
        """Per-kernel device ms of the last timed evaluation (see include/spider.h)
        and the number of events the minibatch touched."""
        ms = (C.c_float * 10)()
        ev = C.c_int64()
        _check(load_library().spider_last_kernel_timing(self.h, ms, C.byref(ev)), self.h)
        names = ["select_pairs", "travel_time", "k_resid", "k_merge_rhs", "whitening", "k_final",
                 "k_merge_s", "centroid", "k_event", "logpost"]
        return dict(zip(names, list(ms))), ev.value

    def spider_last_whiten_timing(self):
        """Device ms of the whitening phases of the last timed evaluation (see
        include/spider.h); zeros unless it took the piece-inverse path."""
        ms = (C.c_float * 6)()
        _check(load_library().spider_last_whiten_timing(self.h, ms), self.h)
        names = ["pieces", "unit_setup", "unit_rounds", "cta_passes", "clean_wait", "general"]
        return dict(zip(names, list(ms)))

    def spider_set_wait_limit_ns(self, limit_ns: int):
        _check(load_library().spider_set_wait_limit_ns(self.h, int(limit_ns)), self.h)

    def spider_set_timing(self, on: bool):
        _check(load_library().spider_set_timing(self.h, 1 if on else 0), self.h)

    def spider_last_timing(self):
        ms = (C.c_float * 5)()
        pairs, nobs, it = C.c_int64(), C.c_int64(), C.c_int32()
        _check(load_library().spider_last_timing(self.h, ms, C.byref(pairs), C.byref(nobs),
                                                 C.byref(it)), self.h)
        return dict(ms=list(ms), pairs=pairs.value, n_obs=nobs.value, pcg_iters=it.value)

    def spider_set_tuning(self, knobs):
        arr = np.ascontiguousarray(knobs, dtype=np.int32)
        _check(load_library().spider_set_tuning(self.h, _ptr(arr, C.c_int32), arr.size), self.h)

    def spider_info(self):
        out = np.zeros(39, np.int64)
        _check(load_library().spider_info(self.h, _ptr(out, C.c_int64), 39), self.h)
        keys = ["n_sub", "graph", "blocks_per_step", "blocks", "pairs", "events", "obs", "components",
                "local_nodes", "piece_inverses", "piece_whitening", "units", "fallback", "units_global",
                "unit_kcycles_shared", "unit_kcycles_global"]
        keys += [f"pass{p}_{n}" for p in range(3) for n in ("setup", "ginv", "sinv", "rounds", "units")]
        keys += [f"handover_{n}" for n in ("pieces", "shared_occ", "shared_nodes", "piece_shared", "ginv_fail",
                                           "sinv_fail", "pool")]
        keys += ["graph_kernels"]
        return dict(zip(keys, (int(x) for x in out)))

    def spider_diagnostics(self, batch_seed: int, eps: float):
        norms = np.empty(self.M, np.float64)
        ratio = C.c_double()
        _check(load_library().spider_diagnostics(self.h, C.c_uint64(batch_seed), C.c_float(eps),
                                                 _ptr(norms, C.c_double), C.byref(ratio)), self.h)
        return norms, ratio.value

    def spider_debug_blocks(self, cap: int = 1 << 20):
        out = np.empty(cap, np.int64)
        n = C.c_int64()
        _check(load_library().spider_debug_blocks(self.h, _ptr(out, C.c_int64), cap, C.byref(n)), self.h)
        return out[: min(cap, n.value)]

    def spider_debug_obs(self, cap: int):
        idx = np.empty(cap, np.int64)
        r = np.empty(cap, np.float32)
        q = np.empty(cap, np.float32)
        n = C.c_int64()
        _check(load_library().spider_debug_obs(self.h, _ptr(idx, C.c_int64), _ptr(r, C.c_float),
                                               _ptr(q, C.c_float), cap, C.byref(n)), self.h)
        k = min(cap, n.value)
        return idx[:k], r[:k], q[:k]


def spider_philox_words(seed: int, c0: int, c1: int, c2: int, c3: int, n: int) -> np.ndarray:
    out = np.empty((n, 4), np.uint32)
    code = load_library().spider_philox_words(C.c_uint64(seed), c0, c1, c2, c3, n,
                                              _ptr(out, C.c_uint32))
    _check(code, None)
    return out


class NetDevice:
    """A network uploaded for spider_tt_pairs (spider_net_upload / spider_net_free)."""

    def __init__(self, net: Net, precision: int = FP32):
        h = C.c_void_p()
        _check(load_library().spider_net_upload(C.byref(net.s), precision, C.byref(h)), None)
        self.h = h
        self.net = net

    def close(self):
        if getattr(self, "h", None):
            load_library().spider_net_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spider_tt_pairs(self, P: int, src_ptr: int, rcv_ptr: int, thi_ptr: int, tlo_ptr: int,
                        j_ptr: int, stream: int = 0):
        """Device pointers (ints) in, device results out; see include/spider.h."""
        _check(load_library().spider_tt_pairs(self.h, P, C.c_void_p(src_ptr), C.c_void_p(rcv_ptr),
                                              C.c_void_p(thi_ptr), C.c_void_p(tlo_ptr or None),
                                              C.c_void_p(j_ptr or None), C.c_void_p(stream or None)),
               None)


def spider_tt_pairs_noalloc(net: Net, P: int, src_ptr: int, rcv_ptr: int, thi_ptr: int,
                            tlo_ptr: int = 0, j_ptr: int = 0, stream: int = 0):
    """Allocation-free travel times (see include/spider.h): host network,
    device inputs and outputs given as integer pointers."""
    code = load_library().spider_tt_pairs_noalloc(
        C.byref(net.s), P, C.c_void_p(src_ptr), C.c_void_p(rcv_ptr), C.c_void_p(thi_ptr),
        C.c_void_p(tlo_ptr or None), C.c_void_p(j_ptr or None), C.c_void_p(stream or None))
    _check(code, None)
