"""ctypes binding of the C-ABI in ``include/rankfhe.h`` (argument marshalling only).

Every operation runs in the CUDA library ``_lib/librankfhe.so``; there is no
fallback.  Importing this module loads the library and raises ``ImportError`` if
it has not been built (``python -m paper_2412_15126_gb300.build`` or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librankfhe.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
_L = ctypes.CDLL(LIB_PATH)

RK_OK, RK_EINVAL, RK_ENOMEM, RK_EDEPTH, RK_ETIMEOUT, RK_ECUDA, RK_EFORMAT, RK_ENOKEY = range(8)
STATUS_NAMES = {0: "RK_OK", 1: "RK_EINVAL", 2: "RK_ENOMEM", 3: "RK_EDEPTH", 4: "RK_ETIMEOUT",
                5: "RK_ECUDA", 6: "RK_EFORMAT", 7: "RK_ENOKEY"}
LAYOUT_ROW, LAYOUT_COL = 0, 1
MASK_ROW0, MASK_COL0, MASK_TIE, MASK_TRI, MASK_VALID = 1, 2, 3, 4, 5
KEY_RELIN, KEY_GALOIS = 1, 2
TIES_CORRECT = 1
TIES_FIRST, TIES_ALL = 0, 2
MASK_ROW0S, MASK_COL0S, MASK_TIEC, MASK_SORTIDX, MASK_ROWIDX = 6, 7, 8, 9, 10
OPT_KS_FUSED, OPT_KS_GROUP_BYTES, OPT_BLOCK_STACKING = 1, 2, 3
OPT_TRIM_LEVELS = 4
OPT_SERVER_LANES = 5
OPT_PAIR_PACKING = 6
OPT_STACK_BUDGET, OPT_INDICATOR_BUDGET = 7, 8
OPT_NTT_GROUP_BYTES, OPT_MODUP_COL = 9, 10
OP_RANK, OP_ORDER_STAT, OP_SORT, OP_RANK_BLOCKED, OP_ORDER_STAT_BLOCKED, OP_SORT_BLOCKED = 1, 2, 3, 4, 5, 6


class RkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint32) for name in
                ("log_n", "n_limbs", "n_special", "digit_size", "log_scale", "log_q0", "log_special", "d_g", "d_f",
                 "cmp_cheb", "prime_form")]


_vp = ctypes.c_void_p
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32 = ctypes.c_uint32
_sz = ctypes.c_size_t


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_L, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("rk_ctx_create", [ctypes.POINTER(Params), ctypes.c_int, _vp, ctypes.POINTER(_vp)])
_sig("rk_ctx_destroy", [_vp], None)
_sig("rk_ctx_moduli", [_vp, _u64p, _sz, ctypes.POINTER(_sz)])
_sig("rk_ctx_scales", [_vp, _dp, _sz])
_sig("rk_sync", [_vp])
_sig("rk_ctx_counters", [_vp, _u64p])
_sig("rk_ctx_set_option", [_vp, _u32, ctypes.c_int64])
_sig("rk_autotune", [_vp, _dp, _sz, ctypes.POINTER(_sz)])
_sig("rk_keygen", [_vp, ctypes.c_uint64, _u32])
_sig("rk_keygen_rotations", [_vp, _i32p, _sz])
_sig("rk_secret_import", [_vp, _i64p, _sz])
_sig("rk_key_import", [_vp, _u32, ctypes.c_uint64, _u64p, _sz])
_sig("rk_key_import_seeded", [_vp, _u32, ctypes.c_uint64, ctypes.c_uint64, _u64p, _sz])
_sig("rk_galois_left", [_vp, ctypes.c_int32], ctypes.c_uint64)
_sig("rk_encoding_import", [_vp, _u32, _u32, _u32, _u32, _dp, _sz])
_sig("rk_encoding_export", [_vp, _u32, _u32, _u32, _u32, _dp, _sz])
_sig("rk_indicator_export", [_vp, _u32, _dp, _sz, ctypes.POINTER(_sz)])
_sig("rk_comparator_export", [_vp, _dp, _sz, ctypes.POINTER(_sz)])
_sig("rk_measure_alu", [_vp, _dp])
_sig("rk_params_chain", [ctypes.POINTER(Params), _u64p, _sz, ctypes.POINTER(_sz), _dp, _sz])
_sig("rk_device_alloc_count", [], ctypes.c_uint64)
_sig("rk_encrypt", [_vp, _dp, _u32, _u32, _u32, _u32, ctypes.POINTER(_vp)])
_sig("rk_decrypt_slots", [_vp, _vp, _dp, _sz])
_sig("rk_decrypt", [_vp, _vp, _dp, _sz, ctypes.POINTER(_u32)])
_sig("rk_ct_import", [_vp, _u64p, _u32, _u32, _u32, _u32, ctypes.POINTER(_vp)])
_sig("rk_ct_export", [_vp, _u64p, _sz])
_sig("rk_ct_level", [_vp], _u32)
_sig("rk_ct_free", [_vp], None)
_sig("rk_ct_stack", [_vp, ctypes.POINTER(_vp), _u32, ctypes.POINTER(_vp)])
_sig("rk_rank_blocked", [_vp, ctypes.POINTER(_vp), _u32, _u32, ctypes.POINTER(_vp)])
_sig("rk_ct_unstack", [_vp, _vp, ctypes.POINTER(_vp)])
_sig("rk_order_stat_blocked", [_vp, ctypes.POINTER(_vp), _u32, _u32, _u32, ctypes.POINTER(_vp)])
_sig("rk_rank_blocked_partial", [_vp, ctypes.POINTER(_vp), _u32, ctypes.POINTER(_u32), ctypes.POINTER(_u32), _u32,
                                 ctypes.POINTER(_vp), ctypes.POINTER(_vp)])
_sig("rk_rank_blocked_finish", [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _u32, ctypes.POINTER(_vp)])
_sig("rk_sort_blocked", [_vp, ctypes.POINTER(_vp), _u32, _u32, ctypes.POINTER(_vp)])
_sig("rk_ct_count", [_vp], _u32)
_sig("rk_rotate", [_vp, _vp, ctypes.c_int32, ctypes.POINTER(_vp)])
_sig("rk_rotate_many", [_vp, _vp, _i32p, _u32, ctypes.POINTER(_vp)])
for _n in ("rk_add", "rk_sub", "rk_mul"):
    _sig(_n, [_vp, _vp, _vp, ctypes.POINTER(_vp)])
_sig("rk_add_const", [_vp, _vp, ctypes.c_double, ctypes.POINTER(_vp)])
_sig("rk_mul_scalar", [_vp, _vp, ctypes.c_double, ctypes.POINTER(_vp)])
_sig("rk_mul_mask", [_vp, _vp, _u32, ctypes.POINTER(_vp)])
_sig("rk_rescale", [_vp, _vp, ctypes.POINTER(_vp)])
_sig("rk_rescale_noalloc", [_vp, _vp, _vp, _u32])
_sig("rk_rank", [_vp, _vp, _u32, ctypes.POINTER(_vp)])
_sig("rk_compare_matrix", [_vp, _vp, ctypes.POINTER(_vp)])
_sig("rk_order_stat", [_vp, _vp, _u32, _u32, ctypes.POINTER(_vp)])
_sig("rk_sort", [_vp, _vp, _u32, ctypes.POINTER(_vp)])
_sig("rk_order_value", [_vp, _vp, _u32, ctypes.POINTER(_vp)])
_sig("rk_median", [_vp, _vp, ctypes.POINTER(_vp)])
_sig("rk_order_value_all", [_vp, _vp, _u32, ctypes.POINTER(_vp)])
_sig("rk_indicator_import", [_vp, _u32, _dp, _sz])
_sig("rk_comparator_import", [_vp, _dp, _sz])
_sig("rk_rank_batch", [_vp, ctypes.POINTER(_vp), _sz, _u32, ctypes.POINTER(_vp)])
_sig("rk_order_stat_batch", [_vp, ctypes.POINTER(_vp), _sz, _u32, _u32, ctypes.POINTER(_vp)])
_sig("rk_sort_batch", [_vp, ctypes.POINTER(_vp), _sz, _u32, ctypes.POINTER(_vp)])
_sig("rk_keys_export", [_vp, ctypes.c_void_p, _sz, ctypes.POINTER(_sz)])
_sig("rk_keys_import", [_vp, ctypes.c_void_p, _sz])
_sig("rk_server_start", [_vp, _sz, _u32])
_sig("rk_server_submit", [_vp, _u32, _u32, _u32, _vp, ctypes.POINTER(ctypes.c_uint64)])
_sig("rk_server_wait", [_vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(_vp)])
_sig("rk_server_poll", [_vp, ctypes.c_uint64, ctypes.POINTER(_vp)])
_sig("rk_server_stats", [_vp, _dp])
_sig("rk_server_stats_lanes", [_vp, _dp])
_sig("rk_server_stop", [_vp])
_sig("rk_server_latencies", [_vp, _dp, _sz, ctypes.POINTER(_sz)])
_sig("rk_graph_rank", [_vp, _vp, _u32, ctypes.POINTER(_vp)])
_sig("rk_graph_capture", [_vp, _u32, _u32, _u32, _u32, _vp, ctypes.POINTER(_vp)])
_sig("rk_graph_run", [_vp, _vp, ctypes.POINTER(_vp)])
_sig("rk_graph_free", [_vp], None)
_sig("rk_ntt_forward", [_vp, _vp, _u32, _u32])
_sig("rk_ntt_inverse", [_vp, _vp, _u32, _u32])
_sig("rk_profile_start", [_vp, ctypes.c_char_p])
_sig("rk_profile_stop", [_vp, _dp])
_sig("rk_profile_kind", [_vp, ctypes.c_char_p, _dp])
_sig("rk_profile_pause", [_vp, ctypes.c_int])
_sig("rk_launch_count", [_vp], ctypes.c_uint64)
_sig("rk_last_error", [], ctypes.c_char_p)


def _check(status):
    if status != RK_OK:
        raise RkError(status, _L.rk_last_error().decode(errors="replace"))


def device_alloc_count() -> int:
    """Device allocations the library has made in this process (every context)."""
    return int(_L.rk_device_alloc_count())


def params_chain(log_n, n_limbs, n_special, digit_size, log_scale, log_q0=60, log_special=61, prime_form=0):
    """The moduli (q_0..q_L, then the special primes) and canonical scales of a
    parameter set, computed on the host by the library (no device needed)."""
    prm = Params(log_n, n_limbs, n_special, digit_size, log_scale, log_q0, log_special, 0, 0, 0, prime_form)
    cnt = _sz()
    q = (ctypes.c_uint64 * (n_limbs + n_special))()
    sc = (ctypes.c_double * n_limbs)()
    _check(_L.rk_params_chain(ctypes.byref(prm), q, len(q), ctypes.byref(cnt), sc, len(sc)))
    return [int(x) for x in q[:cnt.value]], [float(x) for x in sc]


def raw(name):
    """The raw ctypes function of a C-ABI entry point."""
    return getattr(_L, name)


def library_path() -> str:
    return LIB_PATH


class Ciphertext:
    def __init__(self, ctx: "Context", handle: int):
        self.ctx = ctx
        self.handle = ctypes.c_void_p(handle)
        ctx._live.add(self)

    @property
    def level(self) -> int:
        return int(_L.rk_ct_level(self.handle))

    def free(self):
        if self.handle and self.handle.value:
            _L.rk_ct_free(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def export(self) -> np.ndarray:
        n = self.ctx.n
        out = np.empty((2, self.level + 1, n), dtype=np.uint64)
        _check(_L.rk_ct_export(self.handle, out.ctypes.data_as(_u64p), out.size))
        return out


class RankGraph:
    """The rank circuit captured as one CUDA graph for one input shape."""

    def __init__(self, ctx: "Context", handle: int):
        self.ctx = ctx
        self.handle = ctypes.c_void_p(handle)
        ctx._live.add(self)

    def run(self, ct: Ciphertext) -> Ciphertext:
        h = _vp()
        _check(_L.rk_graph_run(self.handle, ct.handle, ctypes.byref(h)))
        return Ciphertext(self.ctx, h.value)

    def free(self):
        if self.handle and self.handle.value:
            _L.rk_graph_free(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    def __init__(self, log_n, n_limbs, n_special, digit_size, log_scale, log_q0=60, log_special=61,
                 d_g=4, d_f=2, device=0, stream=None, cmp_cheb=0, prime_form=0):
        self.params = Params(log_n, n_limbs, n_special, digit_size, log_scale, log_q0, log_special, d_g, d_f, cmp_cheb,
                             prime_form)
        h = _vp()
        _check(_L.rk_ctx_create(ctypes.byref(self.params), device, _vp(stream) if stream else None, ctypes.byref(h)))
        self.handle = h
        self.n = 1 << log_n
        self._live = weakref.WeakSet()
        self._server_inputs = {}

    def close(self):
        """Free every ciphertext still alive, then the context."""
        if self.handle and self.handle.value:
            _L.rk_server_stop(self.handle)   # a running server still reads its inputs
            self._server_inputs = {}
            live = list(self._live)
            for obj in live:                 # graphs first: they hold captured buffers
                if isinstance(obj, RankGraph):
                    obj.free()
            for obj in live:
                obj.free()
            _L.rk_ctx_destroy(self.handle)
            self.handle = _vp(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- parameters ----
    def moduli(self) -> list:
        cnt = _sz()
        _check(_L.rk_ctx_moduli(self.handle, None, 0, ctypes.byref(cnt)))
        out = (ctypes.c_uint64 * cnt.value)()
        _check(_L.rk_ctx_moduli(self.handle, out, cnt.value, ctypes.byref(cnt)))
        return [int(x) for x in out]

    def scales(self) -> list:
        L1 = self.params.n_limbs
        out = (ctypes.c_double * L1)()
        _check(_L.rk_ctx_scales(self.handle, out, L1))
        return list(out)

    def sync(self):
        _check(_L.rk_sync(self.handle))

    def counters(self) -> dict:
        out = (ctypes.c_uint64 * 4)()
        _check(_L.rk_ctx_counters(self.handle, out))
        return dict(zip(("key_switch", "rotate", "mul", "rescale"), [int(x) for x in out]))

    def set_option(self, option: int, value: int):
        _check(_L.rk_ctx_set_option(self.handle, option, int(value)))

    def autotune(self) -> dict:
        """Time candidate launch shapes on this device and keep the fastest (results unchanged)."""
        out = (ctypes.c_double * 64)()
        cnt = _sz()
        _check(_L.rk_autotune(self.handle, out, 64, ctypes.byref(cnt)))
        v = list(out[:cnt.value])
        rep = {}
        for i, slot in enumerate([(s, d, p) for s in ("large", "small") for d in ("fwd", "inv") for p in ("row", "col")]):
            rep["ntt_%s_%s_%s" % slot] = {"units": int(v[2 * i]), "us": v[2 * i + 1]}
        rep["ntt_groups"] = {"us": dict(zip(("whole", "96MiB", "64MiB", "32MiB"), v[16:20])),
                             "choice": "whole" if v[20] == 0 else "%d MiB" % v[20]}
        if len(v) > 21:
            rep["ks"] = {"staged_us": v[21], "fused_us": dict(zip(("24MiB", "48MiB", "96MiB"), v[22:25])),
                         "staged_modup_col_us": v[26],
                         "choice": ("staged, ModUp in the column pass" if v[27] else "staged") if v[25] == 0
                         else "fused %d MiB" % v[25]}
        return rep

    # ---- keys ----
    def keygen(self, seed: int, max_len: int):
        _check(_L.rk_keygen(self.handle, seed, max_len))

    def keygen_rotations(self, rs):
        arr = (ctypes.c_int32 * len(rs))(*rs)
        _check(_L.rk_keygen_rotations(self.handle, arr, len(rs)))

    def secret_import(self, s):
        s = np.ascontiguousarray(s, dtype=np.int64)
        _check(_L.rk_secret_import(self.handle, s.ctypes.data_as(_i64p), s.size))

    def key_import(self, kind, galois, data):
        data = np.ascontiguousarray(data, dtype=np.uint64)
        _check(_L.rk_key_import(self.handle, kind, galois, data.ctypes.data_as(_u64p), data.size))


    def key_import_seeded(self, kind, galois, seed, b_parts):
        """A seeded switching key: its b parts ([beta_L][L+1+alpha][n], coefficient
        domain) and the seed its a parts are regenerated from."""
        data = np.ascontiguousarray(b_parts, dtype=np.uint64)
        _check(_L.rk_key_import_seeded(self.handle, kind, galois, int(seed) & (2**64 - 1), data.ctypes.data_as(_u64p), data.size))
    def galois_left(self, r: int) -> int:
        return int(_L.rk_galois_left(self.handle, r))

    def encoding_import(self, kind, N, Q, n_real, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        _check(_L.rk_encoding_import(self.handle, kind, N, Q, n_real, u.ctypes.data_as(_dp), u.size))

    def encoding_export(self, kind, N, Q=1, n_real=0):
        u = np.empty(self.n, dtype=np.float64)
        _check(_L.rk_encoding_export(self.handle, kind, N, Q, n_real, u.ctypes.data_as(_dp), u.size))
        return u

    def _coeffs_export(self, fn, *args):
        cnt = _sz(0)
        _check(fn(self.handle, *args, None, 0, ctypes.byref(cnt)))
        out = np.empty(cnt.value, dtype=np.float64)
        _check(fn(self.handle, *args, out.ctypes.data_as(_dp), out.size, ctypes.byref(cnt)))
        return out

    def measure_alu(self) -> dict:
        """Integer throughput of the device: 32-bit multiply-adds, Shoup modular products
        and forward NTT butterflies a second (register-resident microbenchmarks); the
        last two also with a prime k 2^32 + 1 (``*_k32``)."""
        out = (ctypes.c_double * 5)()
        _check(_L.rk_measure_alu(self.handle, out))
        return {"imad_per_s": out[0], "modmul_per_s": out[1], "butterfly_per_s": out[2],
                "modmul_k32_per_s": out[3], "butterfly_k32_per_s": out[4]}

    def indicator_export(self, N):
        return self._coeffs_export(_L.rk_indicator_export, N)

    def comparator_export(self):
        return self._coeffs_export(_L.rk_comparator_export)

    # ---- client ----
    def encrypt(self, values, N=None, Q=1, n_real=None) -> Ciphertext:
        v = np.ascontiguousarray(values, dtype=np.float64)
        if n_real is None:
            n_real = v.size // Q
        if N is None:
            N = 1 << max(0, (int(n_real) - 1).bit_length())
        h = _vp()
        _check(_L.rk_encrypt(self.handle, v.ctypes.data_as(_dp), v.size, N, Q, n_real, ctypes.byref(h)))
        return Ciphertext(self, h.value)

    def decrypt(self, ct: Ciphertext) -> np.ndarray:
        cnt = _u32()
        _check(_L.rk_decrypt(self.handle, ct.handle, None, 0, ctypes.byref(cnt)))
        out = np.empty(cnt.value, dtype=np.float64)
        _check(_L.rk_decrypt(self.handle, ct.handle, out.ctypes.data_as(_dp), out.size, ctypes.byref(cnt)))
        return out

    def decrypt_slots(self, ct: Ciphertext) -> np.ndarray:
        out = np.empty(self.n // 2, dtype=np.float64)
        _check(_L.rk_decrypt_slots(self.handle, ct.handle, out.ctypes.data_as(_dp), out.size))
        return out

    def ct_import(self, coeffs, level, N=1, Q=1, n_real=None) -> Ciphertext:
        c = np.ascontiguousarray(coeffs, dtype=np.uint64)
        h = _vp()
        _check(_L.rk_ct_import(self.handle, c.ctypes.data_as(_u64p), level, N, Q, N if n_real is None else n_real, ctypes.byref(h)))
        return Ciphertext(self, h.value)

    # ---- operations ----
    def _out(self, fn, *args) -> Ciphertext:
        h = _vp()
        _check(fn(self.handle, *args, ctypes.byref(h)))
        return Ciphertext(self, h.value)

    def rank_blocked(self, blocks, flags=0):
        ins = (_vp * len(blocks))(*[c.handle.value for c in blocks])
        outs = (_vp * len(blocks))()
        _check(_L.rk_rank_blocked(self.handle, ins, len(blocks), flags, outs))
        return [Ciphertext(self, o) for o in outs]

    def rank_blocked_partial(self, blocks, pairs):
        """Part one of the partitioned blocked rank: the comparisons of the listed block
        pairs (i <= j) and the per-block partial sums (A, B), L ciphertexts each."""
        L = len(blocks)
        ins = (_vp * L)(*[c.handle.value for c in blocks])
        pi = (_u32 * max(len(pairs), 1))(*[int(p[0]) for p in pairs])
        pj = (_u32 * max(len(pairs), 1))(*[int(p[1]) for p in pairs])
        A, B = (_vp * L)(), (_vp * L)()
        _check(_L.rk_rank_blocked_partial(self.handle, ins, L, pi, pj, len(pairs), A, B))
        return [Ciphertext(self, a) for a in A], [Ciphertext(self, b) for b in B]

    def rank_blocked_finish(self, A, B):
        """Part two: the blocked ranks from the partial sums over every pair."""
        L = len(A)
        a = (_vp * L)(*[c.handle.value for c in A])
        b = (_vp * L)(*[c.handle.value for c in B])
        outs = (_vp * L)()
        _check(_L.rk_rank_blocked_finish(self.handle, a, b, L, outs))
        return [Ciphertext(self, o) for o in outs]

    def order_stat_blocked(self, blocks, k, flags=0):
        ins = (_vp * len(blocks))(*[c.handle.value for c in blocks])
        outs = (_vp * len(blocks))()
        _check(_L.rk_order_stat_blocked(self.handle, ins, len(blocks), int(k), flags, outs))
        return [Ciphertext(self, o) for o in outs]

    def sort_blocked(self, blocks, flags=0):
        ins = (_vp * len(blocks))(*[c.handle.value for c in blocks])
        outs = (_vp * len(blocks))()
        _check(_L.rk_sort_blocked(self.handle, ins, len(blocks), flags, outs))
        return [Ciphertext(self, o) for o in outs]

    def stack(self, cts):
        ins = (_vp * len(cts))(*[c.handle.value for c in cts])
        h = _vp()
        _check(_L.rk_ct_stack(self.handle, ins, len(cts), ctypes.byref(h)))
        return Ciphertext(self, h.value)

    def unstack(self, ct):
        k = int(_L.rk_ct_count(ct.handle))
        outs = (_vp * k)()
        _check(_L.rk_ct_unstack(self.handle, ct.handle, outs))
        return [Ciphertext(self, o) for o in outs]

    def rotate(self, ct, r):
        return self._out(_L.rk_rotate, ct.handle, int(r))

    def rotate_many(self, ct, rs):
        arr = (ctypes.c_int32 * len(rs))(*rs)
        outs = (_vp * len(rs))()
        _check(_L.rk_rotate_many(self.handle, ct.handle, arr, len(rs), outs))
        return [Ciphertext(self, o) for o in outs]

    def add(self, a, b):
        return self._out(_L.rk_add, a.handle, b.handle)

    def sub(self, a, b):
        return self._out(_L.rk_sub, a.handle, b.handle)

    def mul(self, a, b):
        return self._out(_L.rk_mul, a.handle, b.handle)

    def add_const(self, a, v):
        return self._out(_L.rk_add_const, a.handle, float(v))

    def mul_scalar(self, a, v):
        return self._out(_L.rk_mul_scalar, a.handle, float(v))

    def mul_mask(self, a, kind):
        return self._out(_L.rk_mul_mask, a.handle, kind)

    def rescale(self, a):
        return self._out(_L.rk_rescale, a.handle)

    def compare_matrix(self, ct):
        return self._out(_L.rk_compare_matrix, ct.handle)

    def order_stat(self, ct, k, flags=0):
        return self._out(_L.rk_order_stat, ct.handle, int(k), flags)

    def sort(self, ct, flags=0):
        return self._out(_L.rk_sort, ct.handle, flags)

    def order_value(self, ct, k):
        return self._out(_L.rk_order_value, ct.handle, int(k))

    def order_value_all(self, ct, k):
        """Value of the k-th statistic from the all-ties mask, divided by its weight
        (Goldschmidt); slot 0 of each query."""
        return self._out(_L.rk_order_value_all, ct.handle, int(k))

    def median(self, ct):
        return self._out(_L.rk_median, ct.handle)

    def comparator_import(self, coeffs):
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        _check(_L.rk_comparator_import(self.handle, c.ctypes.data_as(_dp), c.size))

    def indicator_import(self, N, coeffs):
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        _check(_L.rk_indicator_import(self.handle, N, c.ctypes.data_as(_dp), c.size))

    def rescale_noalloc(self, d_in: int, d_out: int, level: int):
        """Rescale between caller-owned device buffers (evaluation domain) with no
        device allocation; see rk_rescale_noalloc in include/rankfhe.h."""
        _check(_L.rk_rescale_noalloc(self.handle, _vp(d_in), _vp(d_out), level))

    def rank(self, ct, flags=0):
        return self._out(_L.rk_rank, ct.handle, flags)

    # ---- serving loop ----
    def server_start(self, mem_budget_bytes: int, max_stack: int = 32):
        _check(_L.rk_server_start(self.handle, int(mem_budget_bytes), int(max_stack)))

    def server_submit(self, op: int, ct: Ciphertext, arg: int = 0, flags: int = 0) -> int:
        t = ctypes.c_uint64()
        _check(_L.rk_server_submit(self.handle, op, int(arg), flags, ct.handle, ctypes.byref(t)))
        self._server_inputs[int(t.value)] = ct       # borrowed until the result is collected
        return int(t.value)

    def server_wait(self, ticket: int, timeout_s: float = -1.0):
        """The finished request's result, or None while it is pending after timeout_s."""
        h = _vp()
        try:
            _check(_L.rk_server_wait(self.handle, ticket, float(timeout_s), ctypes.byref(h)))
        except RkError:
            self._server_inputs.pop(ticket, None)
            raise
        if not h.value:
            return None
        self._server_inputs.pop(ticket, None)
        return Ciphertext(self, h.value)


    def server_poll(self, ticket: int):
        """The finished request's result, or None while it is pending (no waiting)."""
        return self.server_wait(ticket, 0.0)
    def server_stats(self) -> dict:
        out = (ctypes.c_double * 8)()
        _check(_L.rk_server_stats(self.handle, out))
        keys = ("finished", "p50_s", "p99_s", "max_s", "batches", "mean_batch", "peak_bytes", "queued")
        return dict(zip(keys, list(out)))

    def server_stats_lanes(self) -> dict:
        out = (ctypes.c_double * 5)()
        _check(_L.rk_server_stats_lanes(self.handle, out))
        return {"lanes": int(out[0]), "max_lanes_busy": int(out[1]), "mean_lanes_busy": out[2],
                "packed_requests": int(out[3]), "lane_scratch_bytes": out[4]}

    def server_latencies(self) -> list:
        cnt = _sz()
        _check(_L.rk_server_latencies(self.handle, None, 0, ctypes.byref(cnt)))
        out = (ctypes.c_double * max(cnt.value, 1))()
        _check(_L.rk_server_latencies(self.handle, out, cnt.value, ctypes.byref(cnt)))
        return list(out[:cnt.value])

    def server_stop(self):
        _check(_L.rk_server_stop(self.handle))
        self._server_inputs = {}

    def graph_capture(self, op: int, template: Ciphertext, arg: int = 0, flags: int = 0, L: int = 1) -> RankGraph:
        """Capture the circuit `op` (OP_*) for template-shaped inputs as one CUDA graph;
        blocked circuits take a stack of L blocks and replay to the stack of L results."""
        h = _vp()
        _check(_L.rk_graph_capture(self.handle, op, int(arg), flags, L, template.handle, ctypes.byref(h)))
        return RankGraph(self, h.value)

    def graph_rank(self, template: Ciphertext, flags=0) -> RankGraph:
        """Capture rank(template-shaped input, flags) as one CUDA graph."""
        h = _vp()
        _check(_L.rk_graph_rank(self.handle, template.handle, flags, ctypes.byref(h)))
        return RankGraph(self, h.value)

    def order_stat_batch(self, cts, k, flags=0):
        ins = (_vp * len(cts))(*[c.handle.value for c in cts])
        outs = (_vp * len(cts))()
        _check(_L.rk_order_stat_batch(self.handle, ins, len(cts), int(k), flags, outs))
        return [Ciphertext(self, o) for o in outs]

    def sort_batch(self, cts, flags=0):
        ins = (_vp * len(cts))(*[c.handle.value for c in cts])
        outs = (_vp * len(cts))()
        _check(_L.rk_sort_batch(self.handle, ins, len(cts), flags, outs))
        return [Ciphertext(self, o) for o in outs]

    def keys_export(self) -> np.ndarray:
        """Every switching key as one blob (uint64 words); see rk_keys_export."""
        size = _sz()
        _check(_L.rk_keys_export(self.handle, None, 0, ctypes.byref(size)))
        blob = np.empty(size.value // 8, dtype=np.uint64)
        _check(_L.rk_keys_export(self.handle, blob.ctypes.data, size.value, ctypes.byref(size)))
        return blob

    def keys_import(self, blob: np.ndarray):
        b = np.ascontiguousarray(blob, dtype=np.uint64)
        _check(_L.rk_keys_import(self.handle, b.ctypes.data, b.nbytes))

    def rank_batch(self, cts, flags=0):
        ins = (_vp * len(cts))(*[c.handle.value for c in cts])
        outs = (_vp * len(cts))()
        _check(_L.rk_rank_batch(self.handle, ins, len(cts), flags, outs))
        return [Ciphertext(self, o) for o in outs]

    def profile_start(self, kind):
        _check(_L.rk_profile_start(self.handle, kind.encode() if kind else None))

    def profile_pause(self, paused: bool):
        """Suspend or resume the timing started by profile_start (no synchronisation)."""
        _check(_L.rk_profile_pause(self.handle, 1 if paused else 0))

    def profile_stop(self) -> dict:
        out = (ctypes.c_double * 4)()
        _check(_L.rk_profile_stop(self.handle, out))
        return {"ms": out[0], "launches": int(out[1]), "bytes": out[2], "ops": out[3]}

    def profile_kind(self, kind) -> dict:
        out = (ctypes.c_double * 4)()
        _check(_L.rk_profile_kind(self.handle, kind.encode(), out))
        return {"ms": out[0], "launches": int(out[1]), "bytes": out[2], "ops": out[3]}

    def launch_count(self) -> int:
        return int(_L.rk_launch_count(self.handle))

    def ntt_forward(self, dev_ptr: int, limbs: int, first_prime: int):
        _check(_L.rk_ntt_forward(self.handle, _vp(dev_ptr), limbs, first_prime))

    def ntt_inverse(self, dev_ptr: int, limbs: int, first_prime: int):
        _check(_L.rk_ntt_inverse(self.handle, _vp(dev_ptr), limbs, first_prime))
