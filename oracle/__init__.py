"""EP-HDC CPU oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.

Plain, slow, obviously-correct CPU reference for the client-side inference path of
"Hyperdimensional Computing with Encrypted Parameters" (EP-HDC).  The arithmetic
lives in ``ephdc_oracle.c`` (plain C, exact integers); this module only marshals
numpy arrays and calls the steps in the order the paper gives them:

  Sec. 2.1  random-projection HDC encoding, Sec. 5.1 quantisation to b bits
  Sec. 3    SIMD representation: element d of many query HVs per plaintext
  Sec. 2.2  BFV batch encoding (packing) into slots mod t
  Sec. 4.1  client-side HE: plaintext x encrypted-class-HV multiply-accumulate
  Sec. 2.2/2.3  Galois rotation with key switching (rotate-and-sum over D-chunks)
  (check)   server-side decryption of the similarity scores

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32, u64, i32, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
        vp = ctypes.c_void_p
        sig = {
            "or_is_prime": (ctypes.c_int, [u32]),
            "or_find_primes": (ctypes.c_int, [u32, u32, vp]),
            "or_root_2n": (u32, [u32, u32]),
            "or_quarter_round": (None, [vp]),
            "or_chacha20_block": (None, [vp, u32, vp, vp]),
            "or_stream_words": (None, [u64, u32, u64, u64, u64, vp]),
            "or_cdt_table": (None, [dbl, vp]),
            "or_sample_ternary": (None, [u64, u32, vp]),
            "or_sample_uniform": (None, [u64, u32, u64, u32, u32, vp, vp]),
            "or_sample_gauss": (None, [u64, u32, u64, u32, vp, vp]),
            "or_negacyclic_mul_schoolbook": (None, [u32, u32, vp, vp, vp]),
            "or_ntt": (None, [u32, u32, u32, vp]),
            "or_intt": (None, [u32, u32, u32, vp]),
            "or_polymul": (None, [u32, u32, u32, vp, vp, vp]),
            "or_automorphism": (None, [u32, u32, u32, vp, vp]),
            "or_slot_encode": (None, [u32, u32, u32, vp, vp]),
            "or_slot_decode": (None, [u32, u32, u32, vp, vp]),
            "or_slot_encode_definition": (None, [u32, u32, u32, vp, vp]),
            "or_ctx_size": (ctypes.c_size_t, []),
            "or_ctx_init": (ctypes.c_int, [vp, u32, u32, u32, u32, u32, u32, dbl]),
            "or_ctx_init2": (ctypes.c_int, [vp, u32, u32, u32, u32, u32, u32, dbl, u32, u32,
                                            u32, u32]),
            "or_find_primes_bits": (ctypes.c_int, [u32, u32, u32, vp]),
            "or_ctx_get": (u32, [vp, ctypes.c_int]),
            "or_ctx_cdt": (None, [vp, vp]),
            "or_fold_galois": (u32, [vp, u32]),
            "or_keygen": (None, [vp, u64, vp, vp]),
            "or_encrypt_model": (None, [vp, u64, vp, vp, vp]),
            "or_encrypt_model_seeded_ntt": (None, [vp, u64, vp, vp, vp]),
            "or_seeded_ntt_c1": (None, [vp, u64, u64, vp]),
            "or_hdc_encode": (None, [vp, vp, i32, u32, u32, i32, u32, vp]),
            "or_encode_plain": (None, [vp, vp, i32, vp]),
            "or_ptct_mac": (None, [vp, vp, i32, vp, vp]),
            "or_rotate": (None, [vp, u32, vp, vp]),
            "or_rotate_sum": (None, [vp, vp, i32, vp]),
            "or_decrypt": (None, [vp, vp, vp, vp]),
            "or_decrypt_scores": (None, [vp, vp, vp, i32, vp]),
            "or_decrypt_slots": (None, [vp, vp, vp, vp]),
            "or_encrypt_slots": (None, [vp, u64, u64, vp, vp, vp]),
            "or_noise_budget": (dbl, [vp, vp, vp]),
            "or_encrypt_queries": (None, [vp, u64, vp, i32, vp, vp]),
            "or_encode_model_plain": (None, [vp, vp, vp]),
            "or_ctpt_mac": (None, [vp, vp, i32, vp, vp]),
            "or_num_threads": (ctypes.c_int, []),
            "or_set_threads": (None, [ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _p(a):
    """Pointer of a C-contiguous numpy array."""
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


T = 65537


# ---------------------------------------------------------------- number theory
def is_prime(v):
    return bool(lib().or_is_prime(int(v)))


def find_primes(n, L, bits=30):
    out = np.zeros(L, np.uint32)
    if lib().or_find_primes_bits(n, L, bits, _p(out)):
        raise ValueError("not enough primes")
    return out


def root_2n(p, n):
    return int(lib().or_root_2n(p, n))


def num_threads():
    return int(lib().or_num_threads())


def set_threads(k):
    lib().or_set_threads(int(k))


# ---------------------------------------------------------------- ChaCha20 / samplers
def quarter_round(a, b, c, d):
    x = np.array([a, b, c, d], np.uint32)
    lib().or_quarter_round(_p(x))
    return [int(v) for v in x]


def chacha20_block(key, counter, nonce):
    k = _u32(key)
    nn = _u32(nonce)
    out = np.zeros(16, np.uint32)
    lib().or_chacha20_block(_p(k), counter, _p(nn), _p(out))
    return out


def stream_words(seed, domain, obj, first, count):
    out = np.zeros(count, np.uint32)
    lib().or_stream_words(seed, domain, obj, first, count, _p(out))
    return out


def cdt_table(sigma=3.2):
    T_ = np.zeros(38, np.uint64)
    lib().or_cdt_table(sigma, _p(T_))
    return T_


def sample_ternary(seed, n):
    s = np.zeros(n, np.int32)
    lib().or_sample_ternary(seed, n, _p(s))
    return s


def sample_uniform(seed, domain, obj, n, q):
    q = _u32(q)
    a = np.zeros((len(q), n), np.uint32)
    lib().or_sample_uniform(seed, domain, obj, n, len(q), _p(q), _p(a))
    return a


def sample_gauss(seed, domain, obj, n, sigma=3.2):
    T_ = cdt_table(sigma)
    e = np.zeros(n, np.int32)
    lib().or_sample_gauss(seed, domain, obj, n, _p(T_), _p(e))
    return e


# ---------------------------------------------------------------- polynomials
def negacyclic_mul_schoolbook(a, b, p):
    a, b = _u32(a), _u32(b)
    out = np.zeros_like(a)
    lib().or_negacyclic_mul_schoolbook(len(a), p, _p(a), _p(b), _p(out))
    return out


def ntt(a, p, psi):
    a = _u32(a).copy()
    lib().or_ntt(len(a), p, psi, _p(a))
    return a


def intt(a, p, psi):
    a = _u32(a).copy()
    lib().or_intt(len(a), p, psi, _p(a))
    return a


def polymul(a, b, p, psi):
    a, b = _u32(a), _u32(b)
    out = np.zeros_like(a)
    lib().or_polymul(len(a), p, psi, _p(a), _p(b), _p(out))
    return out


def automorphism(a, g, p):
    a = _u32(a)
    out = np.zeros_like(a)
    lib().or_automorphism(len(a), p, g, _p(a), _p(out))
    return out


def slot_encode(slots, zeta, t=T):
    s = _u32(slots)
    m = np.zeros_like(s)
    lib().or_slot_encode(len(s), t, zeta, _p(s), _p(m))
    return m


def slot_decode(m, zeta, t=T):
    m = _u32(m)
    s = np.zeros_like(m)
    lib().or_slot_decode(len(m), t, zeta, _p(m), _p(s))
    return s


def slot_encode_definition(slots, zeta, t=T):
    s = _u32(slots)
    m = np.zeros_like(s)
    lib().or_slot_encode_definition(len(s), t, zeta, _p(s), _p(m))
    return m


def hdc_encode(X, Wt, shift, bits):
    """Sec. 2.1 random projection A = X Wt^T, then Sec. 5.1 quantisation."""
    X = np.ascontiguousarray(X, np.int8)
    Wt = np.ascontiguousarray(Wt, np.int8)
    B, F = X.shape
    D = Wt.shape[0]
    assert Wt.shape[1] == F
    H = np.zeros((B, D), np.int8)
    lib().or_hdc_encode(_p(X), _p(Wt), B, F, D, shift, bits, _p(H))
    return H


# ---------------------------------------------------------------- BFV context
class Oracle:
    """BFV parameters + (k_in, r) slot layout, and the client path step by step."""

    def __init__(self, n, L, k, k_in, r, D, sigma=3.2, t=T, prime_bits=30, scale_shift=0,
                 scale_group=512):
        self._buf = ctypes.create_string_buffer(lib().or_ctx_size())
        self.ctx = ctypes.cast(self._buf, ctypes.c_void_p)
        if lib().or_ctx_init2(self.ctx, n, L, k, k_in, r, D, sigma, t, prime_bits, scale_shift,
                              scale_group):
            raise ValueError("invalid oracle parameters")
        self.scale_shift, self.scale_group = scale_shift, scale_group
        self.prime_bits = prime_bits
        self.scale_u = int(lib().or_ctx_get(self.ctx, 14))
        g = lambda w: int(lib().or_ctx_get(self.ctx, w))
        self.n, self.L, self.t, self.k, self.k_in, self.r, self.D = (g(i) for i in range(7))
        self.W, self.cap_row, self.cap, self.P, self.Kp, self.logr, self.zeta = (
            g(i) for i in range(7, 14))
        self.q = [g(100 + l) for l in range(self.L)]
        self.psi = [g(200 + l) for l in range(self.L)]
        self.delta = [g(300 + l) for l in range(self.L)]
        self.sigma = sigma

    def groups(self, B):
        return (B + self.cap - 1) // self.cap

    def fold_galois(self, j):
        return int(lib().or_fold_galois(self.ctx, j))

    def ct_words(self):
        return 2 * self.L * self.n

    # server: keys and encrypted model -----------------------------------------
    def keygen(self, seed):
        s = np.zeros(self.n, np.int32)
        gk = np.zeros((max(self.logr, 1), self.L, 2, self.L, self.n), np.uint32)
        lib().or_keygen(self.ctx, seed, _p(s), _p(gk))
        return s, gk[: self.logr]

    def encrypt_model(self, seed, classes, s):
        classes = np.ascontiguousarray(classes, np.int8)
        assert classes.shape == (self.k, self.D)
        model = np.zeros((self.P, self.Kp, 2, self.L, self.n), np.uint32)
        lib().or_encrypt_model(self.ctx, seed, _p(classes), _p(np.ascontiguousarray(s, np.int32)),
                               _p(model))
        return model

    def encrypt_model_seeded_ntt(self, seed, classes, s):
        """The compact model whose c1 is regenerated in the evaluation domain (domain 8,
        word l*n + brv(j) at evaluation psi^(2j+1)); the whole model in the coefficient
        domain, like encrypt_model."""
        classes = np.ascontiguousarray(classes, np.int8)
        assert classes.shape == (self.k, self.D)
        model = np.zeros((self.P, self.Kp, 2, self.L, self.n), np.uint32)
        lib().or_encrypt_model_seeded_ntt(self.ctx, seed, _p(classes),
                                          _p(np.ascontiguousarray(s, np.int32)), _p(model))
        return model

    def seeded_ntt_c1(self, seed, cidx):
        a = np.zeros((self.L, self.n), np.uint32)
        lib().or_seeded_ntt_c1(self.ctx, seed, cidx, _p(a))
        return a

    def encrypt_slots(self, seed, obj, s, slots):
        ct = np.zeros((2, self.L, self.n), np.uint32)
        lib().or_encrypt_slots(self.ctx, seed, obj, _p(np.ascontiguousarray(s, np.int32)),
                               _p(_u32(slots)), _p(ct))
        return ct

    # client path -------------------------------------------------------------
    def encode_plain(self, H):
        H = np.ascontiguousarray(H, np.int8)
        B = H.shape[0]
        assert H.shape[1] == self.D
        m = np.zeros((self.groups(B), self.P, self.n), np.uint32)
        lib().or_encode_plain(self.ctx, _p(H), B, _p(m))
        return m

    def ptct_mac(self, m, B, model):
        m = _u32(m)
        acc = np.zeros((self.groups(B), self.Kp, 2, self.L, self.n), np.uint32)
        lib().or_ptct_mac(self.ctx, _p(m), B, _p(_u32(model)), _p(acc))
        return acc

    def rotate(self, g, gkj, ct):
        ct = _u32(ct).copy()
        lib().or_rotate(self.ctx, g, _p(_u32(gkj)), _p(ct))
        return ct

    def rotate_sum(self, gk, acc):
        acc = _u32(acc).copy()
        count = acc.size // self.ct_words()
        if self.logr:
            lib().or_rotate_sum(self.ctx, _p(_u32(gk)), count, _p(acc))
        return acc

    def infer(self, X, Wt, model, gk, shift, bits):
        """The whole client path S1..S8 for one batch; returns (H, m, out_ct)."""
        H = hdc_encode(X, Wt, shift, bits)
        m = self.encode_plain(H)
        acc = self.ptct_mac(m, H.shape[0], model)
        out = self.rotate_sum(gk, acc)
        return H, m, out

    # server-side variant (HE-HDC-SR, Sec. 3) -----------------------------------
    def encrypt_queries(self, seed, H, s):
        """Client side of the server-side method: every query plaintext encrypted."""
        H = np.ascontiguousarray(H, np.int8)
        B = H.shape[0]
        ctq = np.zeros((self.groups(B), self.P, 2, self.L, self.n), np.uint32)
        lib().or_encrypt_queries(self.ctx, seed, _p(H), B, _p(np.ascontiguousarray(s, np.int32)),
                                 _p(ctq))
        return ctq

    def encode_model_plain(self, classes):
        mm = np.zeros((self.Kp, self.P, self.n), np.uint32)
        lib().or_encode_model_plain(self.ctx, _p(np.ascontiguousarray(classes, np.int8)), _p(mm))
        return mm

    def ctpt_mac(self, ctq, B, mm):
        acc = np.zeros((self.groups(B), self.Kp, 2, self.L, self.n), np.uint32)
        lib().or_ctpt_mac(self.ctx, _p(_u32(ctq)), B, _p(_u32(mm)), _p(acc))
        return acc

    # noise growth (Sec. 5.2, Alg. 1 findDmax) ---------------------------------
    def find_dmax_trial(self, m, model, s, H, cls):
        """One trial of findDmax (one class, r = 1, one group): D_i grows while the
        evaluation with D_i + 1 dimensions decrypts to the clear dot products mod t
        for every query (at most the context's D).  The evaluation with D'
        dimensions is the accumulator sum_{i < D'} lift(m_i) * ct_i; modular
        addition does not depend on the order, so it is built one product at a
        time and decrypted after each."""
        assert self.k == 1 and self.k_in == 1 and self.r == 1
        B = H.shape[0]
        acc = np.zeros((1, 1, 2, self.L, self.n), np.uint32)
        clear = np.zeros(B, np.int64)
        t = self.t
        for i in range(self.D):
            mi = m[0, i].astype(np.int64)
            lm = np.where(mi <= (t - 1) // 2, mi, mi - t)
            for l, p in enumerate(self.q):
                for poly in range(2):
                    prod = polymul(lm % p, model[i, 0, poly, l], p, self.psi[l])
                    acc[0, 0, poly, l] = (acc[0, 0, poly, l].astype(np.int64) + prod) % p
            clear = (clear + H[:, i].astype(np.int64) * int(cls[0, i])) % t
            got = self.decrypt_scores(s, acc, B)[:, 0]
            if not np.array_equal(got, clear.astype(np.uint32)):
                return i
        return self.D

    # server check ------------------------------------------------------------
    def decrypt(self, s, ct):
        out = np.zeros(self.n, np.uint32)
        lib().or_decrypt(self.ctx, _p(np.ascontiguousarray(s, np.int32)), _p(_u32(ct)), _p(out))
        return out

    def decrypt_slots(self, s, ct):
        out = np.zeros(self.n, np.uint32)
        lib().or_decrypt_slots(self.ctx, _p(np.ascontiguousarray(s, np.int32)), _p(_u32(ct)),
                               _p(out))
        return out

    def decrypt_scores(self, s, out_ct, B):
        scores = np.zeros((B, self.k), np.uint32)
        lib().or_decrypt_scores(self.ctx, _p(np.ascontiguousarray(s, np.int32)), _p(_u32(out_ct)),
                                B, _p(scores))
        return scores

    def noise_budget(self, s, ct):
        return float(lib().or_noise_budget(self.ctx, _p(np.ascontiguousarray(s, np.int32)),
                                           _p(_u32(ct))))


def clear_scores(H, classes, t=T):
    """The plain definition the encrypted path reaches: sum_d h[d] c_j[d] mod t."""
    A = np.asarray(H, np.int64) @ np.asarray(classes, np.int64).T
    return np.mod(A, t).astype(np.uint32)
