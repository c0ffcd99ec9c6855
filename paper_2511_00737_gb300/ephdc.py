"""Thin Python binding of the EP-HDC C ABI (include/ephdc.h).

Argument marshalling only: every step of the inference path runs in the CUDA
kernels of ``libephdc.so``.  PyTorch provides device memory and streams; tensors
are passed as raw device pointers.  The functions keep the C names
(``hdc_encode``, ``bfv_encode_plain``, ``bfv_ptct_similarity``,
``bfv_decrypt_scores``, ...); :class:`Context` bundles them with allocation of
correctly sized tensors.  There is no CPU fallback: if the library cannot be built
or loaded, every call raises.
"""
import ctypes
import os

import torch

from . import build as _build

EPHDC_OK = 0
_STATUS = {0: "EPHDC_OK", -1: "EPHDC_EINVAL", -2: "EPHDC_EUNSUPPORTED", -3: "EPHDC_ENOMEM",
           -4: "EPHDC_ECUDA", -5: "EPHDC_ETIMEOUT", -6: "EPHDC_EBUSY"}


class EphdcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class ephdc_request(ctypes.Structure):
    _fields_ = [("X_dev", ctypes.c_void_p), ("B", ctypes.c_int32)]


class ephdc_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("L", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("k_in", ctypes.c_uint32), ("r", ctypes.c_uint32), ("D", ctypes.c_uint32),
                ("F", ctypes.c_uint32), ("hv_bits", ctypes.c_uint32), ("shift", ctypes.c_int32),
                ("max_batch", ctypes.c_uint32), ("sigma", ctypes.c_double),
                ("t", ctypes.c_uint32), ("prime_bits", ctypes.c_uint32),
                ("scale_shift", ctypes.c_uint32), ("scale_group", ctypes.c_uint32)]


_LIB = None
_VP = ctypes.c_void_p
_SIGS = {
    "ephdc_ctx_create": (ctypes.c_int, [ctypes.POINTER(ephdc_params), ctypes.POINTER(_VP)]),
    "ephdc_ctx_destroy": (None, [_VP]),
    "ephdc_last_error": (ctypes.c_char_p, [_VP]),
    "ephdc_query": (ctypes.c_uint64, [_VP, ctypes.c_char_p]),
    "ephdc_sk_bytes": (ctypes.c_size_t, [_VP]),
    "ephdc_galois_key_bytes": (ctypes.c_size_t, [_VP]),
    "ephdc_model_bytes": (ctypes.c_size_t, [_VP]),
    "ephdc_plain_bytes": (ctypes.c_size_t, [_VP, ctypes.c_int32]),
    "ephdc_out_ct_bytes": (ctypes.c_size_t, [_VP, ctypes.c_int32]),
    "bfv_keygen": (ctypes.c_int, [_VP, ctypes.c_uint64, _VP, _VP, _VP]),
    "bfv_encrypt_model": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_uint64, _VP, _VP]),
    "bfv_decrypt_scores": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, _VP, _VP]),
    "hdc_encode": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, _VP, _VP]),
    "bfv_encode_plain": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _VP, _VP]),
    "bfv_ptct_similarity": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _VP, _VP, _VP, _VP]),
    "ephdc_infer": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, _VP, _VP, _VP, _VP]),
    "ephdc_ct_to_host_coeff": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _VP]),
    "ephdc_sk_to_host": (ctypes.c_int, [_VP, _VP, _VP]),
    "ephdc_gk_to_host_coeff": (ctypes.c_int, [_VP, _VP, _VP]),
    "ephdc_plain_to_host_coeff": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _VP]),
    "ephdc_model_to_host_coeff": (ctypes.c_int, [_VP, _VP, _VP]),
    "ephdc_ntt_natural": (ctypes.c_int, [_VP, ctypes.c_uint32, _VP, ctypes.c_int32, ctypes.c_int,
                                         _VP]),
    "bfv_ptct_similarity_noalloc": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _VP, _VP, _VP,
                                                    _VP]),
    "ephdc_device_status": (ctypes.c_int, [_VP]),
    "ephdc_wait_selfcheck": (ctypes.c_int, [_VP, ctypes.c_int64, _VP]),
    "ephdc_infer_multi": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP]),
    "ephdc_tune_set": (ctypes.c_int, [_VP, ctypes.c_char_p, ctypes.c_int64]),
    "ephdc_tune_get": (ctypes.c_int64, [_VP, ctypes.c_char_p]),
    "ephdc_profile_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "ephdc_profile_read": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ephdc_query_ct_bytes": (ctypes.c_size_t, [_VP, ctypes.c_int32]),
    "ephdc_model_plain_bytes": (ctypes.c_size_t, [_VP]),
    "bfv_encrypt_queries": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _VP, ctypes.c_uint64, _VP,
                                           _VP]),
    "bfv_encode_model_plain": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "bfv_ctpt_similarity": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _VP, _VP, _VP, _VP]),
    "ephdc_measure_int_peaks": (ctypes.c_int, [_VP, _VP]),
    "ephdc_find_dmax_trial": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, _VP, _VP, _VP, _VP]),
    "ephdc_model_seeded_bytes": (ctypes.c_size_t, [_VP]),
    "bfv_model_to_seeded": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "bfv_model_to_digits": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "bfv_model_from_seeded": (ctypes.c_int, [_VP, _VP, ctypes.c_uint64, _VP, _VP]),
}

STAGES = ["hdc_encode", "encode_plain", "mac", "rotate", "export", "encrypt_queries"]


def lib_path():
    return _build.LIB


def lib():
    """Load libephdc.so (building it in-tree with nvcc if it is missing or stale)."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def exported_symbols():
    return list(_SIGS)


# ------------------------------------------------------------------ marshalling
def _ptr(t, name, nbytes=None, dtype=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if nbytes is not None and t.numel() * t.element_size() < nbytes:
        raise ValueError("%s holds %d bytes, needs %d" % (name, t.numel() * t.element_size(),
                                                          nbytes))
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(ctx, status):
    if status != EPHDC_OK:
        msg = lib().ephdc_last_error(ctx)
        raise EphdcError(status, msg.decode() if msg else "")


# ------------------------------------------------------------------ C names
def ephdc_ctx_create(n, L, k, k_in, r, D, F, hv_bits, shift, max_batch, sigma=3.2, t=0,
                     prime_bits=0, scale_shift=0, scale_group=0):
    p = ephdc_params(n, L, k, k_in, r, D, F, hv_bits, shift, max_batch, sigma, t, prime_bits,
                     scale_shift, scale_group)
    out = _VP()
    st = lib().ephdc_ctx_create(ctypes.byref(p), ctypes.byref(out))
    _check(None, st)
    return out


def ephdc_ctx_destroy(ctx):
    lib().ephdc_ctx_destroy(ctx)


def bfv_keygen(ctx, seed, sk, gk, stream=None):
    _check(ctx, lib().bfv_keygen(ctx, seed, _ptr(sk, "sk"), _ptr(gk, "gk"), _stream(stream)))


def bfv_encrypt_model(ctx, classes, sk, seed, model, stream=None):
    _check(ctx, lib().bfv_encrypt_model(ctx, _ptr(classes, "classes", dtype=torch.int8),
                                        _ptr(sk, "sk"), seed, _ptr(model, "model"),
                                        _stream(stream)))


def bfv_decrypt_scores(ctx, sk, out_ct, B, scores, stream=None):
    _check(ctx, lib().bfv_decrypt_scores(ctx, _ptr(sk, "sk"), _ptr(out_ct, "out_ct"), B,
                                         _ptr(scores, "scores"), _stream(stream)))


def hdc_encode(ctx, X, Wt, B, H, stream=None):
    _check(ctx, lib().hdc_encode(ctx, _ptr(X, "X", dtype=torch.int8),
                                 _ptr(Wt, "Wt", dtype=torch.int8), B,
                                 _ptr(H, "H", dtype=torch.int8), _stream(stream)))


def bfv_encode_plain(ctx, H, B, pt, stream=None):
    _check(ctx, lib().bfv_encode_plain(ctx, _ptr(H, "H", dtype=torch.int8), B, _ptr(pt, "pt"),
                                       _stream(stream)))


def bfv_ptct_similarity(ctx, pt, B, model, gk, out_ct, stream=None):
    _check(ctx, lib().bfv_ptct_similarity(ctx, _ptr(pt, "pt"), B, _ptr(model, "model"),
                                          _ptr(gk, "gk"), _ptr(out_ct, "out_ct"),
                                          _stream(stream)))


def bfv_ptct_similarity_noalloc(ctx, pt, B, model, gk, out_ct, stream=None):
    """bfv_ptct_similarity with its scratch in the library's fixed device array: for
    callers that must not allocate device memory while serving."""
    _check(ctx, lib().bfv_ptct_similarity_noalloc(ctx, _ptr(pt, "pt"), B, _ptr(model, "model"),
                                                  _ptr(gk, "gk"), _ptr(out_ct, "out_ct"),
                                                  _stream(stream)))


def ephdc_infer(ctx, X, Wt, B, model, gk, out_ct, stream=None):
    _check(ctx, lib().ephdc_infer(ctx, _ptr(X, "X", dtype=torch.int8),
                                  _ptr(Wt, "Wt", dtype=torch.int8), B, _ptr(model, "model"),
                                  _ptr(gk, "gk"), _ptr(out_ct, "out_ct"), _stream(stream)))


def ephdc_infer_multi(ctx, Xs, Wt, model, gk, out_ct, stream=None):
    """Xs: list of int8 CUDA tensors [B_r][F] (one per client), packed back to back."""
    arr = (ephdc_request * len(Xs))()
    for r, X in enumerate(Xs):
        B = X.shape[0]
        arr[r].X_dev = _ptr(X, "X", dtype=torch.int8) if B else None
        arr[r].B = B
    _check(ctx, lib().ephdc_infer_multi(ctx, arr, len(Xs), _ptr(Wt, "Wt", dtype=torch.int8),
                                        _ptr(model, "model"), _ptr(gk, "gk"),
                                        _ptr(out_ct, "out_ct"), _stream(stream)))


# server-side variant (HE-HDC-SR): the client encrypts its queries
def bfv_encrypt_queries(ctx, H, B, sk, seed, query_ct, stream=None):
    _check(ctx, lib().bfv_encrypt_queries(ctx, _ptr(H, "H", dtype=torch.int8), B, _ptr(sk, "sk"),
                                          seed, _ptr(query_ct, "query_ct"), _stream(stream)))


def bfv_encode_model_plain(ctx, classes, model_plain, stream=None):
    _check(ctx, lib().bfv_encode_model_plain(ctx, _ptr(classes, "classes", dtype=torch.int8),
                                             _ptr(model_plain, "model_plain"), _stream(stream)))


def bfv_ctpt_similarity(ctx, query_ct, B, model_plain, gk, out_ct, stream=None):
    _check(ctx, lib().bfv_ctpt_similarity(ctx, _ptr(query_ct, "query_ct"), B,
                                          _ptr(model_plain, "model_plain"), _ptr(gk, "gk"),
                                          _ptr(out_ct, "out_ct"), _stream(stream)))


def ephdc_find_dmax_trial(ctx, sk, H, classes, pt, model):
    """Largest D' <= D whose evaluations with 1..D' dimensions all decrypt correctly."""
    out = ctypes.c_int32(0)
    _check(ctx, lib().ephdc_find_dmax_trial(ctx, _ptr(sk, "sk"), _ptr(H, "H", dtype=torch.int8),
                                            H.shape[0], _ptr(classes, "classes", dtype=torch.int8),
                                            _ptr(pt, "pt"), _ptr(model, "model"),
                                            ctypes.byref(out)))
    return out.value


def ephdc_measure_int_peaks():
    """(butterflies/s, 64-bit multiply-accumulates/s) of the current device."""
    b, m = ctypes.c_double(0), ctypes.c_double(0)
    _check(None, lib().ephdc_measure_int_peaks(ctypes.byref(b), ctypes.byref(m)))
    return b.value, m.value


# ------------------------------------------------------------------ convenience
class Context:
    """One set of BFV parameters + slot layout; allocates correctly sized tensors."""

    def __init__(self, n, L, k, k_in, r, D, F, hv_bits, shift, max_batch, sigma=3.2,
                 device=None, t=0, prime_bits=0, scale_shift=0, scale_group=0):
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.ctx = ephdc_ctx_create(n, L, k, k_in, r, D, F, hv_bits, shift, max_batch, sigma,
                                        t, prime_bits, scale_shift, scale_group)
        self.n, self.L, self.k, self.k_in, self.r, self.D, self.F = n, L, k, k_in, r, D, F
        self.hv_bits, self.shift, self.max_batch = hv_bits, shift, max_batch
        q = lambda w: int(lib().ephdc_query(self.ctx, w.encode()))
        self.cap, self.P, self.Kp, self.W, self.logr = q("cap"), q("P"), q("Kp"), q("W"), q("logr")
        self.q = [q("q%d" % l) for l in range(L)]
        self.t = q("t")

    @classmethod
    def for_workload(cls, w, max_batch=None):
        return cls(w.n, w.L, w.k, w.k_in, w.r, w.D, w.F, w.bits, w.shift,
                   max_batch or max(1, w.B))

    def close(self):
        if self.ctx:
            ephdc_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, what):
        return int(lib().ephdc_query(self.ctx, what.encode()))

    def groups(self, B):
        return (B + self.cap - 1) // self.cap

    def _u32(self, nbytes):
        return torch.empty(nbytes // 4, dtype=torch.int32, device=self.device)

    # allocation + call helpers
    def keygen(self, seed, stream=None):
        sk = self._u32(lib().ephdc_sk_bytes(self.ctx))
        gkb = lib().ephdc_galois_key_bytes(self.ctx)
        gk = self._u32(gkb) if gkb else None
        bfv_keygen(self.ctx, seed, sk, gk, stream)
        return sk, gk

    def encrypt_model(self, classes, sk, seed, stream=None):
        model = self._u32(lib().ephdc_model_bytes(self.ctx))
        bfv_encrypt_model(self.ctx, classes, sk, seed, model, stream)
        return model

    def hdc_encode(self, X, Wt, stream=None):
        B = X.shape[0]
        H = torch.empty((B, self.D), dtype=torch.int8, device=self.device)
        hdc_encode(self.ctx, X, Wt, B, H, stream)
        return H

    def encode_plain(self, H, stream=None):
        B = H.shape[0]
        pt = self._u32(lib().ephdc_plain_bytes(self.ctx, B))
        bfv_encode_plain(self.ctx, H, B, pt, stream)
        return pt

    def out_ct(self, B):
        return self._u32(lib().ephdc_out_ct_bytes(self.ctx, B))

    def ptct_similarity(self, pt, B, model, gk, stream=None):
        out = self.out_ct(B)
        bfv_ptct_similarity(self.ctx, pt, B, model, gk, out, stream)
        return out

    def ptct_similarity_into(self, pt, B, model, gk, out, stream=None):
        bfv_ptct_similarity(self.ctx, pt, B, model, gk, out, stream)
        return out

    def infer(self, X, Wt, model, gk, out=None, stream=None):
        B = X.shape[0]
        out = self.out_ct(B) if out is None else out
        ephdc_infer(self.ctx, X, Wt, B, model, gk, out, stream)
        return out

    # seeded model message (c0 + seed)
    def model_to_seeded(self, model, stream=None):
        out = self._u32(lib().ephdc_model_seeded_bytes(self.ctx))
        _check(self.ctx, lib().bfv_model_to_seeded(self.ctx, _ptr(model, "model"),
                                                   _ptr(out, "seeded"), _stream(stream)))
        return out

    def model_to_digits(self, model, stream=None):
        """The digit model (this context has "model_digits" 1) of a residue model in the
        standard device order."""
        out = self._u32(lib().ephdc_model_bytes(self.ctx))
        _check(self.ctx, lib().bfv_model_to_digits(self.ctx, _ptr(model, "model"),
                                                   _ptr(out, "model_digits"), _stream(stream)))
        return out

    def model_from_seeded(self, seeded, seed, stream=None):
        model = self._u32(lib().ephdc_model_bytes(self.ctx))
        _check(self.ctx, lib().bfv_model_from_seeded(self.ctx, _ptr(seeded, "seeded"), seed,
                                                     _ptr(model, "model"), _stream(stream)))
        return model

    # server-side variant
    def encrypt_queries(self, H, sk, seed, out=None, stream=None):
        B = H.shape[0]
        ctq = self._u32(lib().ephdc_query_ct_bytes(self.ctx, B)) if out is None else out
        bfv_encrypt_queries(self.ctx, H, B, sk, seed, ctq, stream)
        return ctq

    def encode_model_plain(self, classes, stream=None):
        mm = self._u32(lib().ephdc_model_plain_bytes(self.ctx))
        bfv_encode_model_plain(self.ctx, classes, mm, stream)
        return mm

    def ctpt_similarity(self, query_ct, B, model_plain, gk, out=None, stream=None):
        out = self.out_ct(B) if out is None else out
        bfv_ctpt_similarity(self.ctx, query_ct, B, model_plain, gk, out, stream)
        return out

    def decrypt_scores(self, sk, out_ct, B, stream=None):
        scores = torch.empty((B, self.k), dtype=torch.int32, device=self.device)
        bfv_decrypt_scores(self.ctx, sk, out_ct, B, scores, stream)
        return scores

    # host formats (synchronous)
    def ct_to_host_coeff(self, ct, count):
        import numpy as np
        host = np.zeros((count, 2, self.L, self.n), np.uint32)
        _check(self.ctx, lib().ephdc_ct_to_host_coeff(self.ctx, _ptr(ct, "ct"), count,
                                                      host.ctypes.data_as(_VP)))
        return host

    def sk_to_host(self, sk):
        import numpy as np
        host = np.zeros(self.n, np.int32)
        _check(self.ctx, lib().ephdc_sk_to_host(self.ctx, _ptr(sk, "sk"), host.ctypes.data_as(_VP)))
        return host

    def gk_to_host_coeff(self, gk):
        import numpy as np
        host = np.zeros((self.logr, self.L, 2, self.L, self.n), np.uint32)
        if self.logr:
            _check(self.ctx, lib().ephdc_gk_to_host_coeff(self.ctx, _ptr(gk, "gk"),
                                                          host.ctypes.data_as(_VP)))
        return host

    def model_to_host_coeff(self, model):
        import numpy as np
        host = np.zeros((self.P, self.Kp, 2, self.L, self.n), np.uint32)
        _check(self.ctx, lib().ephdc_model_to_host_coeff(self.ctx, _ptr(model, "model"),
                                                         host.ctypes.data_as(_VP)))
        return host

    def plain_to_host_coeff(self, pt, count):
        import numpy as np
        host = np.zeros((count, self.L, self.n), np.uint32)
        _check(self.ctx, lib().ephdc_plain_to_host_coeff(self.ctx, _ptr(pt, "pt"), count,
                                                         host.ctypes.data_as(_VP)))
        return host

    def infer_multi(self, Xs, Wt, model, gk, out=None, stream=None):
        B = sum(int(X.shape[0]) for X in Xs)
        out = self.out_ct(B) if out is None else out
        ephdc_infer_multi(self.ctx, Xs, Wt, model, gk, out, stream)
        return out

    def tune_set(self, knob, value):
        _check(self.ctx, lib().ephdc_tune_set(self.ctx, knob.encode(), int(value)))

    def tune_get(self, knob):
        return int(lib().ephdc_tune_get(self.ctx, knob.encode()))

    def device_status(self):
        """Raise EphdcError(EPHDC_ETIMEOUT) if a bounded device wait gave up."""
        _check(self.ctx, lib().ephdc_device_status(self.ctx))

    def wait_selfcheck(self, limit_cycles, stream=None):
        """Enqueue a kernel whose bounded wait cannot succeed and gives up after
        limit_cycles; the next device_status() raises EPHDC_ETIMEOUT."""
        _check(self.ctx, lib().ephdc_wait_selfcheck(self.ctx, int(limit_cycles),
                                                    _stream(stream)))

    def profile(self, on=True):
        _check(self.ctx, lib().ephdc_profile_enable(self.ctx, 1 if on else 0))

    def profile_read(self):
        """{stage: summed device ms}, {stage: calls}, kernel launches since the last read"""
        import numpy as np
        ms = np.zeros(len(STAGES), np.float64)
        calls = np.zeros(len(STAGES), np.uint64)
        launches = ctypes.c_uint64(0)
        _check(self.ctx, lib().ephdc_profile_read(self.ctx, ms.ctypes.data_as(_VP),
                                                  calls.ctypes.data_as(_VP),
                                                  ctypes.byref(launches)))
        return (dict(zip(STAGES, ms.tolist())), dict(zip(STAGES, calls.tolist())),
                int(launches.value))

    def ntt_natural(self, poly, limb, inverse=False, stream=None):
        count = poly.numel() // self.n
        _check(self.ctx, lib().ephdc_ntt_natural(self.ctx, limb, _ptr(poly, "poly"), count,
                                                 1 if inverse else 0, _stream(stream)))
        return poly
