"""Pure-Python schoolbook BFV for tiny rings -- TEST INFRASTRUCTURE.

A second, independent statement of the oracle's arithmetic, written directly from
the definitions with Python integers and O(n^2) loops, for n <= 64:

* negacyclic products by schoolbook convolution (x^n = -1),
* slot encoding and decoding by direct evaluation at zeta^e over the odd
  exponents e (Sec. 2.2 packing),
* ChaCha20 written again from RFC 8439 Sec. 2.3,
* decryption by the Chinese remainder theorem in Python big integers.

It follows the same conventions as the C oracle (prime choice, root choice, slot
order, PRNG stream layout, (k_in, r) slot layout of Sec. 3) so that the two can
be compared word for word; it shares no code with it.
"""
import math

T = 65537
MASK = 0xFFFFFFFF


# ------------------------------------------------------------------ number theory
def is_prime(v):
    if v < 2:
        return False
    f = 2
    while f * f <= v:
        if v % f == 0:
            return False
        f += 1
    return True


def primes(n, L):
    out, j = [], 1
    while len(out) < L:
        c = (1 << 30) - j * 2 * n + 1
        if c <= 1:
            raise ValueError("no more primes")
        if is_prime(c):
            out.append(c)
        j += 1
    return out


def root_2n(p, n):
    x = 2
    while pow(x, (p - 1) // 2, p) != p - 1:
        x += 1
    return pow(x, (p - 1) // (2 * n), p)


# ------------------------------------------------------------------ ChaCha20
def _rotl(v, c):
    return ((v << c) | (v >> (32 - c))) & MASK


def _qr(x, a, b, c, d):
    x[a] = (x[a] + x[b]) & MASK; x[d] = _rotl(x[d] ^ x[a], 16)
    x[c] = (x[c] + x[d]) & MASK; x[b] = _rotl(x[b] ^ x[c], 12)
    x[a] = (x[a] + x[b]) & MASK; x[d] = _rotl(x[d] ^ x[a], 8)
    x[c] = (x[c] + x[d]) & MASK; x[b] = _rotl(x[b] ^ x[c], 7)


def chacha20_block(key, counter, nonce):
    st = [0x61707865, 0x3320646E, 0x79622D32, 0x6B206574] + list(key) + [counter] + list(nonce)
    x = list(st)
    for _ in range(10):
        _qr(x, 0, 4, 8, 12); _qr(x, 1, 5, 9, 13); _qr(x, 2, 6, 10, 14); _qr(x, 3, 7, 11, 15)
        _qr(x, 0, 5, 10, 15); _qr(x, 1, 6, 11, 12); _qr(x, 2, 7, 8, 13); _qr(x, 3, 4, 9, 14)
    return [(x[i] + st[i]) & MASK for i in range(16)]


class Stream:
    """Word w of the (seed, domain, obj) stream: word w%16 of block w//16."""

    def __init__(self, seed, domain, obj):
        self.key = [seed & MASK, (seed >> 32) & MASK] + [0] * 6
        self.nonce = [domain, (obj >> 32) & MASK, obj & MASK]
        self.cache = {}

    def word(self, w):
        b = w // 16
        if b not in self.cache:
            self.cache[b] = chacha20_block(self.key, b, self.nonce)
        return self.cache[b][w % 16]

    def word64(self, k):
        return self.word(2 * k) | (self.word(2 * k + 1) << 32)


def cdt_table(sigma=3.2):
    w = [math.exp(-((x * x) / (2.0 * sigma * sigma))) for x in range(-19, 20)]
    total = 0.0
    for v in w:
        total += v
    out, cum = [], 0.0
    for m in range(38):
        cum += w[m]
        out.append(int(math.ldexp(cum / total, 64)))
    return out


def gauss_poly(seed, domain, obj, n, table):
    st = Stream(seed, domain, obj)
    return [-19 + sum(1 for th in table if st.word64(kk) >= th) for kk in range(n)]


def uniform_poly(seed, domain, obj, n, q):
    st = Stream(seed, domain, obj)
    return [[st.word64(l * n + kk) % p for kk in range(n)] for l, p in enumerate(q)]


def ternary(seed, n):
    st = Stream(seed, 1, 0)
    return [{0: 0, 1: 1, 2: -1}[st.word(kk) % 3] for kk in range(n)]


# ------------------------------------------------------------------ polynomials
def negamul(a, b, p):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            if i + j < n:
                out[i + j] += a[i] * b[j]
            else:
                out[i + j - n] -= a[i] * b[j]
    return [v % p for v in out]


def automorphism(a, g, p):
    n = len(a)
    out = [0] * n
    for kk in range(n):
        d = (kk * g) % (2 * n)
        if d < n:
            out[d] += a[kk]
        else:
            out[d - n] -= a[kk]
    return [v % p for v in out]


def slot_exponents(n):
    """exponent of slot (rho, i) in order rho * n/2 + i"""
    e0 = [pow(3, i, 2 * n) for i in range(n // 2)]
    return e0 + [2 * n - e for e in e0]


def encode(slots, zeta, t=T):
    n = len(slots)
    zinv, ninv = pow(zeta, t - 2, t), pow(n, t - 2, t)
    exps = slot_exponents(n)
    return [ninv * sum(v * pow(zinv, (e * kk) % (2 * n), t) for v, e in zip(slots, exps)) % t
            for kk in range(n)]


def decode(m, zeta, t=T):
    n = len(m)
    return [sum(c * pow(zeta, (e * kk) % (2 * n), t) for kk, c in enumerate(m)) % t
            for e in slot_exponents(n)]


# ------------------------------------------------------------------ BFV
class TinyBFV:
    def __init__(self, n, L, k, k_in, r, D, sigma=3.2):
        assert n <= 64
        self.n, self.L, self.k, self.k_in, self.r, self.D = n, L, k, k_in, r, D
        self.t = T
        self.q = primes(n, L)
        self.Q = 1
        for p in self.q:
            self.Q *= p
        self.zeta = root_2n(T, n)
        self.delta = self.Q // T
        self.W = n // (2 * r)
        self.cap_row = self.W // k_in
        self.cap = 2 * self.cap_row
        self.P = -(-D // r)
        self.Kp = k // k_in
        self.logr = r.bit_length() - 1
        self.table = cdt_table(sigma)

    def fold_galois(self, j):
        return pow(3, self.W << j, 2 * self.n)

    def keygen(self, seed):
        n, L = self.n, self.L
        s = ternary(seed, n)
        gk = []
        for j in range(self.logr):
            g = self.fold_galois(j)
            per_digit = []
            for i in range(L):
                obj = (j << 16) | i
                a = uniform_poly(seed, 4, obj, n, self.q)
                e = gauss_poly(seed, 5, obj, n, self.table)
                k0, k1 = [], []
                for l, p in enumerate(self.q):
                    sl = [v % p for v in s]
                    as_ = negamul(a[l], sl, p)
                    ts = automorphism(sl, g, p)
                    k0.append([(e[kk] - as_[kk] + (ts[kk] if i == l else 0)) % p
                               for kk in range(n)])
                    k1.append(list(a[l]))
                per_digit.append((k0, k1))
            gk.append(per_digit)
        return s, gk

    def _encrypt(self, seed, obj, s, m):
        a = uniform_poly(seed, 2, obj, self.n, self.q)
        e = gauss_poly(seed, 3, obj, self.n, self.table)
        c0, c1 = [], []
        for l, p in enumerate(self.q):
            as_ = negamul(a[l], [v % p for v in s], p)
            # scaled message round(Q m / t), ties up, written with Python integers
            c0.append([(e[kk] - as_[kk] + (self.Q * m[kk] + (T + 1) // 2) // T) % p
                       for kk in range(self.n)])
            c1.append(list(a[l]))
        return (c0, c1)

    def class_slots(self, classes, i, jp):
        n, half = self.n, self.n // 2
        slots = [0] * n
        for rho in range(2):
            for ch in range(self.r):
                d = i * self.r + ch
                if d >= self.D:
                    continue
                for jin in range(self.k_in):
                    v = classes[jp * self.k_in + jin][d] % T
                    for qq in range(self.cap_row):
                        slots[rho * half + ch * self.W + jin * self.cap_row + qq] = v
        return slots

    def query_slots(self, H, g, i):
        n, half, B = self.n, self.n // 2, len(H)
        slots = [0] * n
        for rho in range(2):
            for ch in range(self.r):
                d = i * self.r + ch
                if d >= self.D:
                    continue
                for qq in range(self.cap_row):
                    beta = g * self.cap + rho * self.cap_row + qq
                    if beta >= B:
                        continue
                    for jin in range(self.k_in):
                        slots[rho * half + ch * self.W + jin * self.cap_row + qq] = H[beta][d] % T
        return slots

    def encrypt_model(self, seed, classes, s):
        model = []
        for i in range(self.P):
            row = []
            for jp in range(self.Kp):
                m = encode(self.class_slots(classes, i, jp), self.zeta)
                row.append(self._encrypt(seed, i * self.Kp + jp, s, m))
            model.append(row)
        return model

    def encode_plain(self, H):
        G = -(-len(H) // self.cap)
        return [[encode(self.query_slots(H, g, i), self.zeta) for i in range(self.P)]
                for g in range(G)]

    def lift(self, m, p):
        return [(c if c <= (T - 1) // 2 else c - T) % p for c in m]

    def ptct_mac(self, m, model):
        out = []
        for g in range(len(m)):
            row = []
            for jp in range(self.Kp):
                polys = []
                for poly in range(2):
                    limbs = []
                    for l, p in enumerate(self.q):
                        acc = [0] * self.n
                        for i in range(self.P):
                            pr = negamul(self.lift(m[g][i], p), model[i][jp][poly][l], p)
                            acc = [(x + y) % p for x, y in zip(acc, pr)]
                        limbs.append(acc)
                    polys.append(limbs)
                row.append(tuple(polys))
            out.append(row)
        return out

    def rotate(self, ct, j, gk):
        g = self.fold_galois(j)
        c0 = [automorphism(ct[0][l], g, p) for l, p in enumerate(self.q)]
        c1 = [automorphism(ct[1][l], g, p) for l, p in enumerate(self.q)]
        n0, n1 = [], []
        for l, p in enumerate(self.q):
            acc0, acc1 = list(c0[l]), [0] * self.n
            for i in range(self.L):
                d = [v % p for v in c1[i]]
                k0, k1 = gk[j][i]
                acc0 = [(x + y) % p for x, y in zip(acc0, negamul(d, k0[l], p))]
                acc1 = [(x + y) % p for x, y in zip(acc1, negamul(d, k1[l], p))]
            n0.append(acc0)
            n1.append(acc1)
        return (n0, n1)

    def rotate_sum(self, ct, gk):
        for j in range(self.logr):
            rc = self.rotate(ct, j, gk)
            ct = tuple([[(x + y) % p for x, y in zip(ct[poly][l], rc[poly][l])]
                        for l, p in enumerate(self.q)] for poly in range(2))
        return ct

    def decrypt(self, s, ct):
        xs = []
        for l, p in enumerate(self.q):
            cs = negamul(ct[1][l], [v % p for v in s], p)
            xs.append([(ct[0][l][kk] + cs[kk]) % p for kk in range(self.n)])
        out = []
        for kk in range(self.n):
            x = 0
            for l, p in enumerate(self.q):
                Ql = self.Q // p
                x += xs[l][kk] * pow(Ql, p - 2, p) * Ql
            x %= self.Q
            out.append(((T * x + self.Q // 2) // self.Q) % T)
        return out

    def scores(self, s, out, B):
        sc = [[0] * self.k for _ in range(B)]
        half = self.n // 2
        for g in range(len(out)):
            for jp in range(self.Kp):
                v = decode(self.decrypt(s, out[g][jp]), self.zeta)
                for rho in range(2):
                    for qq in range(self.cap_row):
                        beta = g * self.cap + rho * self.cap_row + qq
                        if beta >= B:
                            continue
                        for jin in range(self.k_in):
                            sc[beta][jp * self.k_in + jin] = v[rho * half + jin * self.cap_row + qq]
        return sc
