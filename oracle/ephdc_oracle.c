/*
 * EP-HDC CPU oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * A plain, slow, deliberately unoptimised CPU implementation of the client-side
 * inference path of "Hyperdimensional Computing with Encrypted Parameters"
 * (EP-HDC): random-projection HDC encoding with quantisation (Sec. 2.1, Sec. 5.1),
 * BFV batch encoding of query hypervectors into SIMD slots (Sec. 2.2, Sec. 3),
 * plaintext x ciphertext multiply-accumulate against the encrypted class
 * hypervectors (Sec. 4.1), Galois rotate-and-sum with key switching (Sec. 2.2,
 * Sec. 2.3) and, for checking, decryption of the similarity scores.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  The CUDA library shares no code, header, table or constant
 * generator with it: both follow the same written conventions independently.
 *
 * All arithmetic is exact integer arithmetic.  The single floating-point step is
 * the cumulative table of the discrete Gaussian (host double precision, exp()).
 *
 * Conventions the paper leaves open (each is a reading; see the design notes):
 *   primes      q_l = l-th largest prime < 2^30 with q_l = 1 (mod 2n)
 *   roots       psi = x^((q-1)/2n), x = least quadratic non-residue >= 2
 *   NTT domain  a_hat[j] = a(psi^(2j+1))                    (natural order here)
 *   slots       slot (rho, i) <-> exponent e = 3^i (rho=0) or 2n-3^i (rho=1)
 *   PRNG        ChaCha20 block function (RFC 8439), key = seed, nonce = (domain, obj)
 *   Gaussian    sigma = 3.2, support [-19, 19], cumulative-table inversion
 *   key switch  BV decomposition over the RNS digits [c1]_{q_i}, no special prime
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint32_t u32;
typedef uint64_t u64;
typedef int32_t i32;
typedef int64_t i64;

#define OR_MAXL 8
#define OR_T 65537u
#define OR_GAUSS_TAIL 19
#define OR_CDT_LEN (2 * OR_GAUSS_TAIL)

/* ------------------------------------------------------------------------- */
/* Modular arithmetic on residues < 2^32 (plain % on 64-bit products).        */
/* ------------------------------------------------------------------------- */
static u32 mulmod(u32 a, u32 b, u32 m) { return (u32)(((u64)a * b) % m); }
static u32 addmod(u32 a, u32 b, u32 m) { return (u32)(((u64)a + b) % m); }
static u32 submod(u32 a, u32 b, u32 m) { return (u32)(((u64)a + m - (b % m)) % m); }
static u32 powmod(u32 b, u64 e, u32 m) {
  u64 r = 1 % m, x = b % m;
  while (e) {
    if (e & 1) r = (r * x) % m;
    x = (x * x) % m;
    e >>= 1;
  }
  return (u32)r;
}
/* inverse modulo a prime (Fermat) */
static u32 invmod(u32 a, u32 p) { return powmod(a, (u64)p - 2, p); }
/* signed integer -> residue in [0, m) */
static u32 smod(i64 v, u32 m) {
  i64 r = v % (i64)m;
  if (r < 0) r += m;
  return (u32)r;
}

/* Deterministic Miller-Rabin: bases 2, 7, 61 decide every n < 4,759,123,141. */
int or_is_prime(u32 n) {
  static const u32 bases[3] = {2, 7, 61};
  if (n < 2) return 0;
  for (int i = 0; i < 3; i++)
    if (n % bases[i] == 0) return n == bases[i];
  u32 d = n - 1;
  int s = 0;
  while ((d & 1) == 0) { d >>= 1; s++; }
  for (int i = 0; i < 3; i++) {
    u64 x = powmod(bases[i], d, n);
    if (x == 1 || x == n - 1) continue;
    int comp = 1;
    for (int r = 1; r < s; r++) {
      x = (x * x) % n;
      if (x == n - 1) { comp = 0; break; }
    }
    if (comp) return 0;
  }
  return 1;
}

/* RNS primes: the L largest primes q < 2^30 with q = 1 (mod 2n), in decreasing
 * order.  Sec. 2.2 needs q = 1 (mod 2n) so that x^n + 1 splits (NTT-friendly). */
int or_find_primes_bits(u32 n, u32 L, u32 bits, u32* q_out) {
  u64 two_n = 2ull * n;
  u32 found = 0;
  for (u64 j = 1; found < L; j++) {
    if (j * two_n >= (1ull << bits)) return -1;
    u32 c = (u32)((1ull << bits) - j * two_n + 1);
    if (or_is_prime(c)) q_out[found++] = c;
  }
  return 0;
}

int or_find_primes(u32 n, u32 L, u32* q_out) { return or_find_primes_bits(n, L, 30, q_out); }

/* Least x >= 2 with x^((p-1)/2) = -1 (a quadratic non-residue, Euler's criterion);
 * psi = x^((p-1)/(2n)) then has order exactly 2n. */
u32 or_root_2n(u32 p, u32 n) {
  u32 x = 2;
  while (powmod(x, (p - 1) / 2, p) != p - 1) x++;
  return powmod(x, (p - 1) / (2ull * n), p);
}

/* ------------------------------------------------------------------------- */
/* ChaCha20 block function, RFC 8439 Sec. 2.3.                                */
/* ------------------------------------------------------------------------- */
static u32 rotl32(u32 v, int c) { return (v << c) | (v >> (32 - c)); }
static void quarter(u32* x, int a, int b, int c, int d) {
  x[a] += x[b]; x[d] ^= x[a]; x[d] = rotl32(x[d], 16);
  x[c] += x[d]; x[b] ^= x[c]; x[b] = rotl32(x[b], 12);
  x[a] += x[b]; x[d] ^= x[a]; x[d] = rotl32(x[d], 8);
  x[c] += x[d]; x[b] ^= x[c]; x[b] = rotl32(x[b], 7);
}
void or_quarter_round(u32* abcd) { quarter(abcd, 0, 1, 2, 3); }

void or_chacha20_block(const u32 key[8], u32 counter, const u32 nonce[3], u32 out[16]) {
  u32 st[16], x[16];
  st[0] = 0x61707865u; st[1] = 0x3320646eu; st[2] = 0x79622d32u; st[3] = 0x6b206574u;
  for (int i = 0; i < 8; i++) st[4 + i] = key[i];
  st[12] = counter;
  st[13] = nonce[0]; st[14] = nonce[1]; st[15] = nonce[2];
  memcpy(x, st, sizeof x);
  for (int r = 0; r < 10; r++) {
    quarter(x, 0, 4, 8, 12); quarter(x, 1, 5, 9, 13);
    quarter(x, 2, 6, 10, 14); quarter(x, 3, 7, 11, 15);
    quarter(x, 0, 5, 10, 15); quarter(x, 1, 6, 11, 12);
    quarter(x, 2, 7, 8, 13); quarter(x, 3, 4, 9, 14);
  }
  for (int i = 0; i < 16; i++) out[i] = x[i] + st[i];
}

/* The counter-based stream of 32-bit words for (seed, domain, obj):
 * key = (lo32 seed, hi32 seed, 0 x 6), nonce = (domain, hi32 obj, lo32 obj),
 * word w = word (w mod 16) of block number floor(w / 16). */
typedef struct {
  u32 key[8], nonce[3];
  u64 cached_block;
  u32 buf[16];
} stream_t;

static void stream_init(stream_t* s, u64 seed, u32 domain, u64 obj) {
  memset(s, 0, sizeof *s);
  s->key[0] = (u32)seed;
  s->key[1] = (u32)(seed >> 32);
  s->nonce[0] = domain;
  s->nonce[1] = (u32)(obj >> 32);
  s->nonce[2] = (u32)obj;
  s->cached_block = ~0ull;
}
static u32 stream_word(stream_t* s, u64 w) {
  u64 blk = w / 16;
  if (blk != s->cached_block) {
    or_chacha20_block(s->key, (u32)blk, s->nonce, s->buf);
    s->cached_block = blk;
  }
  return s->buf[w % 16];
}
/* 64-bit word k = 32-bit words 2k (low half) and 2k+1 (high half). */
static u64 stream_word64(stream_t* s, u64 k) {
  u64 lo = stream_word(s, 2 * k);
  u64 hi = stream_word(s, 2 * k + 1);
  return lo | (hi << 32);
}

void or_stream_words(u64 seed, u32 domain, u64 obj, u64 first, u64 count, u32* out) {
  stream_t s;
  stream_init(&s, seed, domain, obj);
  for (u64 i = 0; i < count; i++) out[i] = stream_word(&s, first + i);
}

/* ------------------------------------------------------------------------- */
/* Samplers (Sec. 2.2: RLWE encryption with ternary secret and Gaussian error) */
/* ------------------------------------------------------------------------- */
/* Cumulative table for the discrete Gaussian on [-19, 19], weights
 * exp(-x^2 / (2 sigma^2)): T[m] = floor(2^64 * P(X <= -19 + m)), m = 0..37. */
void or_cdt_table(double sigma, u64* T) {
  double w[2 * OR_GAUSS_TAIL + 1];
  double total = 0.0;
  for (int x = -OR_GAUSS_TAIL; x <= OR_GAUSS_TAIL; x++) {
    double xx = (double)x * (double)x;
    double den = 2.0 * sigma * sigma;
    w[x + OR_GAUSS_TAIL] = exp(-(xx / den));
  }
  for (int m = 0; m <= 2 * OR_GAUSS_TAIL; m++) total += w[m];
  double cum = 0.0;
  for (int m = 0; m < OR_CDT_LEN; m++) {
    cum += w[m];
    T[m] = (u64)ldexp(cum / total, 64);
  }
}

static i32 cdt_sample(const u64* T, u64 u) {
  i32 c = 0;
  for (int m = 0; m < OR_CDT_LEN; m++)
    if (u >= T[m]) c++;
  return -OR_GAUSS_TAIL + c;
}

/* ternary secret: word kappa mod 3 -> {0 -> 0, 1 -> 1, 2 -> -1}; domain 1, obj 0 */
void or_sample_ternary(u64 seed, u32 n, i32* s_out) {
  stream_t s;
  stream_init(&s, seed, 1, 0);
  for (u32 k = 0; k < n; k++) {
    u32 v = stream_word(&s, k) % 3u;
    s_out[k] = (v == 2) ? -1 : (i32)v;
  }
}

/* uniform polynomial in R_q: limb l coefficient kappa = word64(l*n + kappa) mod q_l */
void or_sample_uniform(u64 seed, u32 domain, u64 obj, u32 n, u32 L, const u32* q, u32* a_out) {
  stream_t s;
  stream_init(&s, seed, domain, obj);
  for (u32 l = 0; l < L; l++)
    for (u32 k = 0; k < n; k++)
      a_out[(u64)l * n + k] = (u32)(stream_word64(&s, (u64)l * n + k) % q[l]);
}

/* Gaussian polynomial: coefficient kappa from word64(kappa) through the table */
void or_sample_gauss(u64 seed, u32 domain, u64 obj, u32 n, const u64* T, i32* e_out) {
  stream_t s;
  stream_init(&s, seed, domain, obj);
  for (u32 k = 0; k < n; k++) e_out[k] = cdt_sample(T, stream_word64(&s, k));
}

/* ------------------------------------------------------------------------- */
/* Polynomial arithmetic in Z_p[x] / (x^n + 1)                                */
/* ------------------------------------------------------------------------- */
/* Definition of the negacyclic product (for pinning the NTT): x^n = -1. */
void or_negacyclic_mul_schoolbook(u32 n, u32 p, const u32* a, const u32* b, u32* out) {
  for (u32 k = 0; k < n; k++) out[k] = 0;
  for (u32 i = 0; i < n; i++)
    for (u32 j = 0; j < n; j++) {
      u32 prod = mulmod(a[i], b[j], p);
      u32 d = i + j;
      if (d < n) out[d] = addmod(out[d], prod, p);
      else out[d - n] = submod(out[d - n], prod, p);
    }
}

static u32 bitrev(u32 v, int bits) {
  u32 r = 0;
  for (int i = 0; i < bits; i++) { r = (r << 1) | (v & 1); v >>= 1; }
  return r;
}
static int log2u(u32 n) { int l = 0; while ((1u << l) < n) l++; return l; }

/* Textbook iterative radix-2 cyclic DFT over Z_p with root w of order n
 * (natural order in, natural order out). */
static void cyclic_dft(u32 n, u32 p, u32 w, u32* a) {
  int lg = log2u(n);
  for (u32 i = 0; i < n; i++) {
    u32 j = bitrev(i, lg);
    if (j > i) { u32 t = a[i]; a[i] = a[j]; a[j] = t; }
  }
  for (u32 len = 2; len <= n; len <<= 1) {
    u32 wl = powmod(w, n / len, p);
    for (u32 st = 0; st < n; st += len) {
      u32 wk = 1;
      for (u32 j = 0; j < len / 2; j++) {
        u32 u = a[st + j];
        u32 v = mulmod(a[st + j + len / 2], wk, p);
        a[st + j] = addmod(u, v, p);
        a[st + j + len / 2] = submod(u, v, p);
        wk = mulmod(wk, wl, p);
      }
    }
  }
}

/* Negacyclic NTT, natural order: a_hat[j] = sum_k a[k] psi^((2j+1)k).
 * Twist by psi^k, then a cyclic DFT with omega = psi^2. */
void or_ntt(u32 n, u32 p, u32 psi, u32* a) {
  u32 pk = 1;
  for (u32 k = 0; k < n; k++) { a[k] = mulmod(a[k], pk, p); pk = mulmod(pk, psi, p); }
  cyclic_dft(n, p, mulmod(psi, psi, p), a);
}

/* Inverse of or_ntt: cyclic inverse DFT, scale by n^-1, untwist by psi^-k. */
void or_intt(u32 n, u32 p, u32 psi, u32* a) {
  u32 psi_inv = invmod(psi, p);
  cyclic_dft(n, p, mulmod(psi_inv, psi_inv, p), a);
  u32 ninv = invmod(n % p, p);
  u32 pk = 1;
  for (u32 k = 0; k < n; k++) {
    a[k] = mulmod(mulmod(a[k], ninv, p), pk, p);
    pk = mulmod(pk, psi_inv, p);
  }
}

/* Negacyclic product through the NTT: INTT(NTT(a) * NTT(b)). */
void or_polymul(u32 n, u32 p, u32 psi, const u32* a, const u32* b, u32* out) {
  u32* fa = (u32*)malloc(sizeof(u32) * n);
  u32* fb = (u32*)malloc(sizeof(u32) * n);
  memcpy(fa, a, sizeof(u32) * n);
  memcpy(fb, b, sizeof(u32) * n);
  or_ntt(n, p, psi, fa);
  or_ntt(n, p, psi, fb);
  for (u32 k = 0; k < n; k++) out[k] = mulmod(fa[k], fb[k], p);
  or_intt(n, p, psi, out);
  free(fa);
  free(fb);
}

/* Galois automorphism tau_g: a(x) -> a(x^g), g odd; x^n = -1 gives the sign. */
void or_automorphism(u32 n, u32 p, u32 g, const u32* a, u32* out) {
  u64 two_n = 2ull * n;
  for (u32 k = 0; k < n; k++) out[k] = 0;
  for (u32 k = 0; k < n; k++) {
    u64 d = ((u64)k * g) % two_n;
    if (d < n) out[d] = addmod(out[d], a[k], p);
    else out[d - n] = submod(out[d - n], a[k], p);
  }
}

/* ------------------------------------------------------------------------- */
/* BFV SIMD slots mod t (batching; Sec. 2.2 "packing")                        */
/* ------------------------------------------------------------------------- */
/* exponent of slot (rho, i): 3^i mod 2n for rho = 0, 2n - 3^i for rho = 1 */
static u32 slot_exponent(u32 n, u32 rho, u32 i) {
  u32 two_n = 2 * n;
  u32 e = powmod(3, i, two_n);
  return rho ? two_n - e : e;
}

/* Encode: m is the unique polynomial of degree < n with m(zeta^e(rho,i)) =
 * slots[rho * n/2 + i].  Place slot values at NTT index (e-1)/2, then INTT. */
void or_slot_encode(u32 n, u32 t, u32 zeta, const u32* slots, u32* m) {
  for (u32 rho = 0; rho < 2; rho++)
    for (u32 i = 0; i < n / 2; i++) {
      u32 e = slot_exponent(n, rho, i);
      m[(e - 1) / 2] = slots[rho * (n / 2) + i] % t;
    }
  or_intt(n, t, zeta, m);
}

/* Decode: slots[rho * n/2 + i] = m(zeta^e(rho,i)). */
void or_slot_decode(u32 n, u32 t, u32 zeta, const u32* m, u32* slots) {
  u32* ev = (u32*)malloc(sizeof(u32) * n);
  memcpy(ev, m, sizeof(u32) * n);
  or_ntt(n, t, zeta, ev);
  for (u32 rho = 0; rho < 2; rho++)
    for (u32 i = 0; i < n / 2; i++) {
      u32 e = slot_exponent(n, rho, i);
      slots[rho * (n / 2) + i] = ev[(e - 1) / 2];
    }
  free(ev);
}

/* O(n^2) definition of the encoder: m_k = n^-1 sum_{odd e} v(e) zeta^(-e k). */
void or_slot_encode_definition(u32 n, u32 t, u32 zeta, const u32* slots, u32* m) {
  u32 zinv = invmod(zeta, t), ninv = invmod(n % t, t);
  u32 two_n = 2 * n;
  for (u32 k = 0; k < n; k++) {
    u32 acc = 0;
    for (u32 rho = 0; rho < 2; rho++)
      for (u32 i = 0; i < n / 2; i++) {
        u32 e = slot_exponent(n, rho, i);
        u32 ex = (u32)(((u64)e * k) % two_n);
        acc = addmod(acc, mulmod(slots[rho * (n / 2) + i] % t, powmod(zinv, ex, t), t), t);
      }
    m[k] = mulmod(acc, ninv, t);
  }
}

/* ------------------------------------------------------------------------- */
/* Small multi-word unsigned integers (base 2^32, little-endian) for q = prod q_l */
/* ------------------------------------------------------------------------- */
#define BW 12 /* words: up to 8 primes of 30 bits, times t, plus headroom */
typedef struct { u32 w[BW]; } big_t;

static void big_zero(big_t* a) { memset(a, 0, sizeof *a); }
static void big_from_u32(big_t* a, u32 v) { big_zero(a); a->w[0] = v; }
static void big_mul_small(big_t* a, u32 m) {
  u64 carry = 0;
  for (int i = 0; i < BW; i++) {
    u64 v = (u64)a->w[i] * m + carry;
    a->w[i] = (u32)v;
    carry = v >> 32;
  }
}
static void big_add(big_t* a, const big_t* b) {
  u64 carry = 0;
  for (int i = 0; i < BW; i++) {
    u64 v = (u64)a->w[i] + b->w[i] + carry;
    a->w[i] = (u32)v;
    carry = v >> 32;
  }
}
static void big_sub(big_t* a, const big_t* b) { /* requires a >= b */
  i64 borrow = 0;
  for (int i = 0; i < BW; i++) {
    i64 v = (i64)a->w[i] - b->w[i] - borrow;
    borrow = v < 0;
    a->w[i] = (u32)(v + (borrow ? (1ll << 32) : 0));
  }
}
static int big_cmp(const big_t* a, const big_t* b) {
  for (int i = BW - 1; i >= 0; i--) {
    if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
  }
  return 0;
}
static void big_shl(big_t* a, int s) { /* s < 32 */
  if (!s) return;
  for (int i = BW - 1; i > 0; i--) a->w[i] = (a->w[i] << s) | (a->w[i - 1] >> (32 - s));
  a->w[0] <<= s;
}
static void big_shr1(big_t* a) {
  for (int i = 0; i < BW - 1; i++) a->w[i] = (a->w[i] >> 1) | (a->w[i + 1] << 31);
  a->w[BW - 1] >>= 1;
}
static u32 big_divmod_small(big_t* a, u32 d) { /* a <- floor(a/d), returns a mod d */
  u64 rem = 0;
  for (int i = BW - 1; i >= 0; i--) {
    u64 cur = (rem << 32) | a->w[i];
    a->w[i] = (u32)(cur / d);
    rem = cur % d;
  }
  return (u32)rem;
}
static u32 big_mod_small(const big_t* a, u32 d) {
  big_t c = *a;
  return big_divmod_small(&c, d);
}

/* ------------------------------------------------------------------------- */
/* BFV context: parameters and the (k_in, r) slot layout                       */
/* ------------------------------------------------------------------------- */
typedef struct {
  u32 n, L, t, k, k_in, r, D;
  u32 W, cap_row, cap, P, Kp, logr;
  u32 q[OR_MAXL], psi[OR_MAXL];
  u32 zeta;
  u32 delta[OR_MAXL]; /* floor(q/t) mod q_l */
  u32 rt;             /* q mod t */
  u64 cdt[OR_CDT_LEN];
  double sigma;
  /* scaling operation (Sec. 5.1): after every scale_group products added to an
   * accumulator, multiply it by scale_u = (2^scale_shift)^-1 mod t; 0 = off */
  u32 scale_shift, scale_group, scale_u;
} or_ctx;

size_t or_ctx_size(void) { return sizeof(or_ctx); }

/* Layout (k_in, r): r D-chunks per plaintext, W = n/(2r) positions per chunk per
 * row, k_in classes side by side inside a chunk, cap_row = floor(W / k_in)
 * queries per row.  r = 1, k_in = k is the paper's SIMD representation
 * (Sec. 3; batch floor(N/k), D plaintexts, no rotation). */
/* t: the plaintext modulus, a prime = 1 (mod 2n) below 2^30 (slot packing needs a
 * primitive 2n-th root of unity mod t); prime_bits: the RNS primes are the L largest
 * primes below 2^prime_bits that are = 1 (mod 2n). */
int or_ctx_init2(or_ctx* c, u32 n, u32 L, u32 k, u32 k_in, u32 r, u32 D, double sigma, u32 t,
                 u32 prime_bits, u32 scale_shift, u32 scale_group) {
  memset(c, 0, sizeof *c);
  if (n < 8 || (n & (n - 1)) || n > 32768) return -1;
  if (L < 1 || L > OR_MAXL || k < 1 || k_in < 1 || k % k_in || D < 1) return -1;
  if (r < 1 || (r & (r - 1)) || r > n / 2) return -1;
  if (t < 3 || t >= (1u << 30) || t % (2 * n) != 1 || !or_is_prime(t)) return -1;
  if (prime_bits < 14 || prime_bits > 30) return -1;
  if (scale_shift > 30 || (scale_shift && scale_group < 1)) return -1;
  c->n = n; c->L = L; c->t = t; c->k = k; c->k_in = k_in; c->r = r; c->D = D;
  c->scale_shift = scale_shift;
  c->scale_group = scale_group;
  /* (2^s)^-1 mod t by Fermat: t is prime */
  c->scale_u = scale_shift ? (u32)powmod((u32)((1ull << scale_shift) % t), t - 2, t) : 1;
  c->sigma = sigma;
  c->W = n / (2 * r);
  c->cap_row = c->W / k_in;
  if (c->cap_row < 1) return -1;
  c->cap = 2 * c->cap_row;
  c->P = (D + r - 1) / r;
  c->Kp = k / k_in;
  c->logr = (u32)log2u(r);
  if (or_find_primes_bits(n, L, prime_bits, c->q)) return -1;
  for (u32 l = 0; l < L; l++) c->psi[l] = or_root_2n(c->q[l], n);
  c->zeta = or_root_2n(t, n);
  /* Delta = floor(q / t), reduced mod each q_l */
  big_t Q;
  big_from_u32(&Q, 1);
  for (u32 l = 0; l < L; l++) big_mul_small(&Q, c->q[l]);
  c->rt = big_divmod_small(&Q, t);
  for (u32 l = 0; l < L; l++) c->delta[l] = big_mod_small(&Q, c->q[l]);
  or_cdt_table(sigma, c->cdt);
  return 0;
}

/* The scaled message of encryption, round(q m / t) with ties up, m in [0, t), reduced
 * mod q_l: q m = (floor(q/t) t + (q mod t)) m, so it is
 * floor(q/t) m + floor(((q mod t) m + floor((t+1)/2)) / t). */
static u32 scaled_msg(const or_ctx* c, u32 l, u32 m) {
  u32 p = c->q[l];
  u64 fix = ((u64)c->rt * m + (c->t + 1) / 2) / c->t;
  return addmod(mulmod(c->delta[l], m, p), (u32)(fix % p), p);
}

int or_ctx_init(or_ctx* c, u32 n, u32 L, u32 k, u32 k_in, u32 r, u32 D, double sigma) {
  return or_ctx_init2(c, n, L, k, k_in, r, D, sigma, OR_T, 30, 0, 512);
}

u32 or_ctx_get(const or_ctx* c, int what) {
  switch (what) {
    case 0: return c->n;   case 1: return c->L;   case 2: return c->t;
    case 3: return c->k;   case 4: return c->k_in; case 5: return c->r;
    case 6: return c->D;   case 7: return c->W;   case 8: return c->cap_row;
    case 9: return c->cap; case 10: return c->P;  case 11: return c->Kp;
    case 12: return c->logr; case 13: return c->zeta;
    case 14: return c->scale_u;
    case 15: return c->rt;
    default: break;
  }
  if (what >= 100 && what < 100 + OR_MAXL) return c->q[what - 100];
  if (what >= 200 && what < 200 + OR_MAXL) return c->psi[what - 200];
  if (what >= 300 && what < 300 + OR_MAXL) return c->delta[what - 300];
  return 0;
}
void or_ctx_cdt(const or_ctx* c, u64* T) { memcpy(T, c->cdt, sizeof c->cdt); }

/* Galois element of rotate-and-sum fold step j: rotate each row left by W*2^j. */
u32 or_fold_galois(const or_ctx* c, u32 j) {
  return powmod(3, (u64)c->W << j, 2 * c->n);
}

/* ------------------------------------------------------------------------- */
/* Key generation (server).  Sec. 2.2: RLWE secret; rotation needs Galois keys. */
/* ------------------------------------------------------------------------- */
/* s: n ternary coefficients.  gk: [logr][L digits][2][L limbs][n] (k0, k1),
 * k1 = a_{j,i}, k0 = -a s + e + delta_{i,l} tau_{g_j}(s) in limb l. */
void or_keygen(const or_ctx* c, u64 seed, i32* s, u32* gk) {
  u32 n = c->n, L = c->L;
  or_sample_ternary(seed, n, s);
  u32* a = (u32*)malloc(sizeof(u32) * L * n);
  i32* e = (i32*)malloc(sizeof(i32) * n);
  u32* sl = (u32*)malloc(sizeof(u32) * n);
  u32* ts = (u32*)malloc(sizeof(u32) * n);
  u32* as = (u32*)malloc(sizeof(u32) * n);
  for (u32 j = 0; j < c->logr; j++) {
    u32 g = or_fold_galois(c, j);
    for (u32 i = 0; i < L; i++) {
      u64 obj = ((u64)j << 16) | i;
      or_sample_uniform(seed, 4, obj, n, L, c->q, a);
      or_sample_gauss(seed, 5, obj, n, c->cdt, e);
      for (u32 l = 0; l < L; l++) {
        u32 p = c->q[l];
        for (u32 kk = 0; kk < n; kk++) sl[kk] = smod(s[kk], p);
        or_automorphism(n, p, g, sl, ts);
        or_polymul(n, p, c->psi[l], a + (u64)l * n, sl, as);
        u32* k0 = gk + ((((u64)j * L + i) * 2 + 0) * L + l) * n;
        u32* k1 = gk + ((((u64)j * L + i) * 2 + 1) * L + l) * n;
        for (u32 kk = 0; kk < n; kk++) {
          u32 v = submod(smod(e[kk], p), as[kk], p);
          if (i == l) v = addmod(v, ts[kk], p);
          k0[kk] = v;
          k1[kk] = a[(u64)l * n + kk];
        }
      }
    }
  }
  free(a); free(e); free(sl); free(ts); free(as);
}

/* ------------------------------------------------------------------------- */
/* Slot layout of query and class hypervectors (Sec. 3 SIMD representation)   */
/* ------------------------------------------------------------------------- */
/* Class plaintext for model ciphertext (i, jp): slot (rho, ch*W + jin*cap_row + qq)
 * holds class (jp*k_in + jin) element d = i*r + ch, for every qq < cap_row.  All
 * other slots (and d >= D) are zero.  classes: [k][D] int8. */
static void class_slots(const or_ctx* c, const int8_t* classes, u32 i, u32 jp, u32* slots) {
  u32 half = c->n / 2;
  memset(slots, 0, sizeof(u32) * c->n);
  for (u32 rho = 0; rho < 2; rho++)
    for (u32 ch = 0; ch < c->r; ch++) {
      u32 d = i * c->r + ch;
      if (d >= c->D) continue;
      for (u32 jin = 0; jin < c->k_in; jin++) {
        u32 cls = jp * c->k_in + jin;
        u32 val = smod(classes[(u64)cls * c->D + d], c->t);
        for (u32 qq = 0; qq < c->cap_row; qq++)
          slots[rho * half + ch * c->W + jin * c->cap_row + qq] = val;
      }
    }
}

/* Query plaintext (g, i): slot (rho, ch*W + jin*cap_row + qq) holds element
 * d = i*r + ch of query beta = g*cap + rho*cap_row + qq, replicated for every
 * jin < k_in (Sec. 3: each query repeated k times).  H: [B][D] int8. */
static void query_slots(const or_ctx* c, const int8_t* H, i32 B, u32 g, u32 i, u32* slots) {
  u32 half = c->n / 2;
  memset(slots, 0, sizeof(u32) * c->n);
  for (u32 rho = 0; rho < 2; rho++)
    for (u32 ch = 0; ch < c->r; ch++) {
      u32 d = i * c->r + ch;
      if (d >= c->D) continue;
      for (u32 qq = 0; qq < c->cap_row; qq++) {
        u64 beta = (u64)g * c->cap + rho * c->cap_row + qq;
        if (beta >= (u64)B) continue;
        u32 val = smod(H[beta * c->D + d], c->t);
        for (u32 jin = 0; jin < c->k_in; jin++)
          slots[rho * half + ch * c->W + jin * c->cap_row + qq] = val;
      }
    }
}

/* ------------------------------------------------------------------------- */
/* Secret-key encryption of the class hypervectors (server, Sec. 4.1)         */
/* ------------------------------------------------------------------------- */
/* model: [P][Kp][2][L][n] coefficient domain.  Ciphertext number cidx = i*Kp + jp:
 * c1 = a (domain 2, obj cidx), c0 = -a s + e (domain 3, obj cidx) + Delta m. */
void or_encrypt_model(const or_ctx* c, u64 seed, const int8_t* classes, const i32* s, u32* model) {
  u32 n = c->n, L = c->L;
#pragma omp parallel
  {
    u32* slots = (u32*)malloc(sizeof(u32) * n);
    u32* m = (u32*)malloc(sizeof(u32) * n);
    u32* a = (u32*)malloc(sizeof(u32) * L * n);
    i32* e = (i32*)malloc(sizeof(i32) * n);
    u32* sl = (u32*)malloc(sizeof(u32) * n);
    u32* as = (u32*)malloc(sizeof(u32) * n);
#pragma omp for schedule(dynamic)
    for (i64 cidx = 0; cidx < (i64)c->P * c->Kp; cidx++) {
      u32 i = (u32)(cidx / c->Kp), jp = (u32)(cidx % c->Kp);
      class_slots(c, classes, i, jp, slots);
      or_slot_encode(n, c->t, c->zeta, slots, m);
      or_sample_uniform(seed, 2, (u64)cidx, n, L, c->q, a);
      or_sample_gauss(seed, 3, (u64)cidx, n, c->cdt, e);
      for (u32 l = 0; l < L; l++) {
        u32 p = c->q[l];
        for (u32 kk = 0; kk < n; kk++) sl[kk] = smod(s[kk], p);
        or_polymul(n, p, c->psi[l], a + (u64)l * n, sl, as);
        u32* c0 = model + (((u64)cidx * 2 + 0) * L + l) * n;
        u32* c1 = model + (((u64)cidx * 2 + 1) * L + l) * n;
        for (u32 kk = 0; kk < n; kk++) {
          u32 v = submod(smod(e[kk], p), as[kk], p);
          v = addmod(v, scaled_msg(c, l, m[kk]), p);
          c0[kk] = v;
          c1[kk] = a[(u64)l * n + kk];
        }
      }
    }
    free(slots); free(m); free(a); free(e); free(sl); free(as);
  }
}

/* The compact model of Sec. 4.1 (the model shipped once): only c0 travels and c1 is
 * regenerated from the seed, here directly in the evaluation domain so that a client
 * can regenerate it while it multiplies.  Convention: c1 of model ciphertext cidx in
 * limb l, evaluated at psi_l^(2j+1), is word64(l*n + brv(j)) mod q_l of the stream
 * (seed, domain 8, cidx), brv reversing the log2 n bits of j (position brv(j) of the
 * evaluation order in which a bit-reversed transform leaves it).  c0 follows the same
 * rule as or_encrypt_model with that c1.  Output: the whole model in the coefficient
 * domain, [P][k/k_in][2][L][n]. */
static u32 bit_reverse(u32 v, u32 bits) {
  u32 r = 0;
  for (u32 b = 0; b < bits; b++) r |= ((v >> b) & 1u) << (bits - 1 - b);
  return r;
}

void or_seeded_ntt_c1(const or_ctx* c, u64 seed, u64 cidx, u32* a_out) {
  u32 n = c->n, logn = 0;
  while ((1u << logn) < n) logn++;
  stream_t s;
  stream_init(&s, seed, 8, cidx);
  for (u32 l = 0; l < c->L; l++) {
    u32* a = a_out + (u64)l * n;
    for (u32 j = 0; j < n; j++)
      a[j] = (u32)(stream_word64(&s, (u64)l * n + bit_reverse(j, logn)) % c->q[l]);
    or_intt(n, c->q[l], c->psi[l], a);  /* evaluations -> coefficients */
  }
}

void or_encrypt_model_seeded_ntt(const or_ctx* c, u64 seed, const int8_t* classes, const i32* s,
                                 u32* model) {
  u32 n = c->n, L = c->L;
#pragma omp parallel
  {
    u32* slots = (u32*)malloc(sizeof(u32) * n);
    u32* m = (u32*)malloc(sizeof(u32) * n);
    u32* a = (u32*)malloc(sizeof(u32) * L * n);
    i32* e = (i32*)malloc(sizeof(i32) * n);
    u32* sl = (u32*)malloc(sizeof(u32) * n);
    u32* as = (u32*)malloc(sizeof(u32) * n);
#pragma omp for schedule(dynamic)
    for (i64 cidx = 0; cidx < (i64)c->P * c->Kp; cidx++) {
      u32 i = (u32)(cidx / c->Kp), jp = (u32)(cidx % c->Kp);
      class_slots(c, classes, i, jp, slots);
      or_slot_encode(n, c->t, c->zeta, slots, m);
      or_seeded_ntt_c1(c, seed, (u64)cidx, a);
      or_sample_gauss(seed, 3, (u64)cidx, n, c->cdt, e);
      for (u32 l = 0; l < L; l++) {
        u32 p = c->q[l];
        for (u32 kk = 0; kk < n; kk++) sl[kk] = smod(s[kk], p);
        or_polymul(n, p, c->psi[l], a + (u64)l * n, sl, as);
        u32* c0 = model + (((u64)cidx * 2 + 0) * L + l) * n;
        u32* c1 = model + (((u64)cidx * 2 + 1) * L + l) * n;
        for (u32 kk = 0; kk < n; kk++) {
          u32 v = submod(smod(e[kk], p), as[kk], p);
          v = addmod(v, scaled_msg(c, l, m[kk]), p);
          c0[kk] = v;
          c1[kk] = a[(u64)l * n + kk];
        }
      }
    }
    free(slots); free(m); free(a); free(e); free(sl); free(as);
  }
}

/* ------------------------------------------------------------------------- */
/* HDC encoding (Sec. 2.1 random projection) and quantisation (Sec. 5.1)       */
/* ------------------------------------------------------------------------- */
/* A[beta][d] = sum_f X[beta][f] * Wt[d][f]  (Wt holds the projection transposed:
 * row d = the weights of dimension d), then
 * h = clamp(floor((A + 2^(shift-1)) / 2^shift), -2^(b-1), 2^(b-1)-1). */
static i64 floor_div_pow2(i64 v, int s) {
  i64 d = (i64)1 << s;
  i64 q = v / d;
  if ((v % d) != 0 && v < 0) q -= 1;
  return q;
}
void or_hdc_encode(const int8_t* X, const int8_t* Wt, i32 B, u32 F, u32 D, i32 shift, u32 bits,
                   int8_t* H) {
  i64 lo = -((i64)1 << (bits - 1)), hi = ((i64)1 << (bits - 1)) - 1;
  i64 half = shift > 0 ? ((i64)1 << (shift - 1)) : 0;
#pragma omp parallel for schedule(static)
  for (i64 b = 0; b < B; b++)
    for (u32 d = 0; d < D; d++) {
      i64 acc = 0;
      for (u32 f = 0; f < F; f++) acc += (i64)X[b * F + f] * (i64)Wt[(u64)d * F + f];
      i64 v = floor_div_pow2(acc + half, shift);
      if (v < lo) v = lo;
      if (v > hi) v = hi;
      H[b * D + d] = (int8_t)v;
    }
}

/* ------------------------------------------------------------------------- */
/* Client: batch-encode the query hypervectors (EncPt)                        */
/* ------------------------------------------------------------------------- */
/* m: [G][P][n] plaintext polynomials mod t (coefficient domain), G = ceil(B/cap). */
void or_encode_plain(const or_ctx* c, const int8_t* H, i32 B, u32* m) {
  u32 n = c->n;
  u32 G = (u32)((B + c->cap - 1) / c->cap);
#pragma omp parallel
  {
    u32* slots = (u32*)malloc(sizeof(u32) * n);
#pragma omp for schedule(dynamic)
    for (i64 gi = 0; gi < (i64)G * c->P; gi++) {
      u32 g = (u32)(gi / c->P), i = (u32)(gi % c->P);
      query_slots(c, H, B, g, i, slots);
      or_slot_encode(n, c->t, c->zeta, slots, m + (u64)gi * n);
    }
    free(slots);
  }
}

/* centred lift of a plaintext coefficient a in [0, t) to (-t/2, t/2], mod p */
static u32 lift(u32 a, u32 t, u32 p) {
  i64 v = (a <= (t - 1) / 2) ? (i64)a : (i64)a - (i64)t;
  return smod(v, p);
}

/* ------------------------------------------------------------------------- */
/* Client: pt x ct multiply-accumulate (HE compute, Sec. 4.1)                 */
/* ------------------------------------------------------------------------- */
/* acc[g][jp][poly][l] = sum_i lift(m[g][i]) * model[i][jp][poly][l] in R_{q_l}. */
void or_ptct_mac(const or_ctx* c, const u32* m, i32 B, const u32* model, u32* acc) {
  u32 n = c->n, L = c->L;
  u32 G = (u32)((B + c->cap - 1) / c->cap);
  i64 jobs = (i64)G * c->Kp * 2 * L;
#pragma omp parallel
  {
    u32* lm = (u32*)malloc(sizeof(u32) * n);
    u32* prod = (u32*)malloc(sizeof(u32) * n);
#pragma omp for schedule(dynamic)
    for (i64 job = 0; job < jobs; job++) {
      u32 l = (u32)(job % L);
      u32 poly = (u32)((job / L) % 2);
      u32 jp = (u32)((job / (2 * L)) % c->Kp);
      u32 g = (u32)(job / (2 * L * c->Kp));
      u32 p = c->q[l];
      u32* out = acc + ((((u64)g * c->Kp + jp) * 2 + poly) * L + l) * n;
      for (u32 kk = 0; kk < n; kk++) out[kk] = 0;
      for (u32 i = 0; i < c->P; i++) {
        const u32* mi = m + ((u64)g * c->P + i) * n;
        for (u32 kk = 0; kk < n; kk++) lm[kk] = lift(mi[kk], c->t, p);
        const u32* ct = model + ((((u64)i * c->Kp + jp) * 2 + poly) * L + l) * n;
        or_polymul(n, p, c->psi[l], lm, ct, prod);
        for (u32 kk = 0; kk < n; kk++) out[kk] = addmod(out[kk], prod[kk], p);
        if (c->scale_shift && (i + 1) % c->scale_group == 0) {
          /* scaling operation: the accumulator times the plaintext scalar
           * (2^s)^-1 mod t, lifted into Z_{q_l} */
          u32 u = lift(c->scale_u, c->t, p);
          for (u32 kk = 0; kk < n; kk++) out[kk] = mulmod(out[kk], u, p);
        }
      }
    }
    free(lm); free(prod);
  }
}

/* ------------------------------------------------------------------------- */
/* Rotation with key switching, and rotate-and-sum (Sec. 2.2, Sec. 2.3)       */
/* ------------------------------------------------------------------------- */
/* ct (in place): [2][L][n].  gkj: Galois key of this step, [L digits][2][L][n].
 * ct' = tau_g(ct); digits d_i = [c1']_{q_i} as integers in [0, q_i);
 * c0'' = c0' + sum_i d_i k0_i,  c1'' = sum_i d_i k1_i. */
void or_rotate(const or_ctx* c, u32 g, const u32* gkj, u32* ct) {
  u32 n = c->n, L = c->L;
  u32* c0r = (u32*)malloc(sizeof(u32) * L * n);
  u32* c1r = (u32*)malloc(sizeof(u32) * L * n);
  u32* dl = (u32*)malloc(sizeof(u32) * n);
  u32* prod = (u32*)malloc(sizeof(u32) * n);
  for (u32 l = 0; l < L; l++) {
    or_automorphism(n, c->q[l], g, ct + (u64)l * n, c0r + (u64)l * n);
    or_automorphism(n, c->q[l], g, ct + ((u64)L + l) * n, c1r + (u64)l * n);
  }
  for (u32 l = 0; l < L; l++) {
    u32 p = c->q[l];
    u32* o0 = ct + (u64)l * n;
    u32* o1 = ct + ((u64)L + l) * n;
    for (u32 kk = 0; kk < n; kk++) { o0[kk] = c0r[(u64)l * n + kk]; o1[kk] = 0; }
    for (u32 i = 0; i < L; i++) {
      const u32* digit = c1r + (u64)i * n;
      for (u32 kk = 0; kk < n; kk++) dl[kk] = digit[kk] % p;
      const u32* k0 = gkj + (((u64)i * 2 + 0) * L + l) * n;
      const u32* k1 = gkj + (((u64)i * 2 + 1) * L + l) * n;
      or_polymul(n, p, c->psi[l], dl, k0, prod);
      for (u32 kk = 0; kk < n; kk++) o0[kk] = addmod(o0[kk], prod[kk], p);
      or_polymul(n, p, c->psi[l], dl, k1, prod);
      for (u32 kk = 0; kk < n; kk++) o1[kk] = addmod(o1[kk], prod[kk], p);
    }
  }
  free(c0r); free(c1r); free(dl); free(prod);
}

/* acc: [count][2][L][n]; for j = 0 .. log2(r)-1: ct <- ct + rotate_{g_j}(ct). */
void or_rotate_sum(const or_ctx* c, const u32* gk, i32 count, u32* acc) {
  u32 n = c->n, L = c->L;
  u64 ctw = 2ull * L * n;
  u64 gkw = (u64)L * 2 * L * n;
#pragma omp parallel
  {
    u32* tmp = (u32*)malloc(sizeof(u32) * ctw);
#pragma omp for schedule(dynamic)
    for (i64 ci = 0; ci < count; ci++) {
      u32* ct = acc + (u64)ci * ctw;
      for (u32 j = 0; j < c->logr; j++) {
        memcpy(tmp, ct, sizeof(u32) * ctw);
        or_rotate(c, or_fold_galois(c, j), gk + (u64)j * gkw, tmp);
        for (u32 l = 0; l < L; l++)
          for (u32 poly = 0; poly < 2; poly++)
            for (u32 kk = 0; kk < n; kk++) {
              u64 idx = ((u64)poly * L + l) * n + kk;
              ct[idx] = addmod(ct[idx], tmp[idx], c->q[l]);
            }
      }
    }
    free(tmp);
  }
}

/* ------------------------------------------------------------------------- */
/* Decryption (server-side check)                                             */
/* ------------------------------------------------------------------------- */
/* m'[k] = round(t * x / q) mod t with x = CRT([c0 + c1 s]_{q_l}) in [0, q);
 * rounding half up: floor((t x + floor(q/2)) / q). */
void or_decrypt(const or_ctx* c, const i32* s, const u32* ct, u32* mout) {
  u32 n = c->n, L = c->L;
  u32* x = (u32*)malloc(sizeof(u32) * L * n);
  u32* sl = (u32*)malloc(sizeof(u32) * n);
  u32* cs = (u32*)malloc(sizeof(u32) * n);
  for (u32 l = 0; l < L; l++) {
    u32 p = c->q[l];
    for (u32 kk = 0; kk < n; kk++) sl[kk] = smod(s[kk], p);
    or_polymul(n, p, c->psi[l], ct + ((u64)L + l) * n, sl, cs);
    for (u32 kk = 0; kk < n; kk++) x[(u64)l * n + kk] = addmod(ct[(u64)l * n + kk], cs[kk], p);
  }
  big_t Q, Qh, Ql[OR_MAXL];
  u32 yinv[OR_MAXL];
  big_from_u32(&Q, 1);
  for (u32 l = 0; l < L; l++) big_mul_small(&Q, c->q[l]);
  Qh = Q;
  big_shr1(&Qh);
  for (u32 l = 0; l < L; l++) {
    big_from_u32(&Ql[l], 1);
    for (u32 o = 0; o < L; o++)
      if (o != l) big_mul_small(&Ql[l], c->q[o]);
    yinv[l] = invmod(big_mod_small(&Ql[l], c->q[l]), c->q[l]);
  }
  for (u32 kk = 0; kk < n; kk++) {
    /* x = sum_l [x_l * (q/q_l)^-1]_{q_l} * (q/q_l), then reduce into [0, q) */
    big_t X;
    big_zero(&X);
    for (u32 l = 0; l < L; l++) {
      big_t term = Ql[l];
      big_mul_small(&term, mulmod(x[(u64)l * n + kk], yinv[l], c->q[l]));
      big_add(&X, &term);
    }
    while (big_cmp(&X, &Q) >= 0) big_sub(&X, &Q);
    /* num = t x + floor(q/2); quotient bit by bit (it is at most t < 2^30) */
    big_t num = X;
    big_mul_small(&num, c->t);
    big_add(&num, &Qh);
    u32 quo = 0;
    for (int b = 30; b >= 0; b--) {
      big_t qs = Q;
      big_shl(&qs, b);
      if (big_cmp(&num, &qs) >= 0) { big_sub(&num, &qs); quo |= 1u << b; }
    }
    mout[kk] = quo % c->t;
  }
  free(x); free(sl); free(cs);
}

/* Scores of queries beta in [0, B): ct layout [G][Kp][2][L][n] after rotate-and-sum;
 * score[beta][jp*k_in + jin] = slot (rho, jin*cap_row + qq) of ct (g, jp),
 * beta = g*cap + rho*cap_row + qq. */
void or_decrypt_scores(const or_ctx* c, const i32* s, const u32* out_ct, i32 B, u32* scores) {
  u32 n = c->n, L = c->L, half = n / 2;
  u32 G = (u32)((B + c->cap - 1) / c->cap);
  u64 ctw = 2ull * L * n;
#pragma omp parallel
  {
    u32* mm = (u32*)malloc(sizeof(u32) * n);
    u32* sv = (u32*)malloc(sizeof(u32) * n);
#pragma omp for schedule(dynamic)
    for (i64 gj = 0; gj < (i64)G * c->Kp; gj++) {
      u32 g = (u32)(gj / c->Kp), jp = (u32)(gj % c->Kp);
      or_decrypt(c, s, out_ct + (u64)gj * ctw, mm);
      or_slot_decode(n, c->t, c->zeta, mm, sv);
      for (u32 rho = 0; rho < 2; rho++)
        for (u32 qq = 0; qq < c->cap_row; qq++) {
          u64 beta = (u64)g * c->cap + rho * c->cap_row + qq;
          if (beta >= (u64)B) continue;
          for (u32 jin = 0; jin < c->k_in; jin++)
            scores[beta * c->k + jp * c->k_in + jin] = sv[rho * half + jin * c->cap_row + qq];
        }
    }
    free(mm); free(sv);
  }
}

/* Plain decrypt of one ciphertext to its slot vector (for pins). */
void or_decrypt_slots(const or_ctx* c, const i32* s, const u32* ct, u32* slots) {
  u32* mm = (u32*)malloc(sizeof(u32) * c->n);
  or_decrypt(c, s, ct, mm);
  or_slot_decode(c->n, c->t, c->zeta, mm, slots);
  free(mm);
}

/* Encrypt an arbitrary slot vector (for pins): same rule as the model, with
 * randomness from (domain 2/3, obj). */
void or_encrypt_slots(const or_ctx* c, u64 seed, u64 obj, const i32* s, const u32* slots, u32* ct) {
  u32 n = c->n, L = c->L;
  u32* m = (u32*)malloc(sizeof(u32) * n);
  u32* a = (u32*)malloc(sizeof(u32) * L * n);
  i32* e = (i32*)malloc(sizeof(i32) * n);
  u32* sl = (u32*)malloc(sizeof(u32) * n);
  u32* as = (u32*)malloc(sizeof(u32) * n);
  u32* sv = (u32*)malloc(sizeof(u32) * n);
  memcpy(sv, slots, sizeof(u32) * n);
  or_slot_encode(n, c->t, c->zeta, sv, m);
  or_sample_uniform(seed, 2, obj, n, L, c->q, a);
  or_sample_gauss(seed, 3, obj, n, c->cdt, e);
  for (u32 l = 0; l < L; l++) {
    u32 p = c->q[l];
    for (u32 kk = 0; kk < n; kk++) sl[kk] = smod(s[kk], p);
    or_polymul(n, p, c->psi[l], a + (u64)l * n, sl, as);
    for (u32 kk = 0; kk < n; kk++) {
      u32 v = submod(smod(e[kk], p), as[kk], p);
      ct[(u64)l * n + kk] = addmod(v, scaled_msg(c, l, m[kk]), p);
      ct[((u64)L + l) * n + kk] = a[(u64)l * n + kk];
    }
  }
  free(m); free(a); free(e); free(sl); free(as); free(sv);
}

/* Noise of a decrypted ciphertext: max_k | t*x_k - q*m'_k | / t expressed as a
 * log2, and the budget log2(q / (2t)) minus that.  Returns the remaining bits. */
double or_noise_budget(const or_ctx* c, const i32* s, const u32* ct) {
  u32 n = c->n, L = c->L;
  u32* x = (u32*)malloc(sizeof(u32) * L * n);
  u32* sl = (u32*)malloc(sizeof(u32) * n);
  u32* cs = (u32*)malloc(sizeof(u32) * n);
  for (u32 l = 0; l < L; l++) {
    u32 p = c->q[l];
    for (u32 kk = 0; kk < n; kk++) sl[kk] = smod(s[kk], p);
    or_polymul(n, p, c->psi[l], ct + ((u64)L + l) * n, sl, cs);
    for (u32 kk = 0; kk < n; kk++) x[(u64)l * n + kk] = addmod(ct[(u64)l * n + kk], cs[kk], p);
  }
  big_t Q, Ql[OR_MAXL];
  u32 yinv[OR_MAXL];
  big_from_u32(&Q, 1);
  for (u32 l = 0; l < L; l++) big_mul_small(&Q, c->q[l]);
  for (u32 l = 0; l < L; l++) {
    big_from_u32(&Ql[l], 1);
    for (u32 o = 0; o < L; o++)
      if (o != l) big_mul_small(&Ql[l], c->q[o]);
    yinv[l] = invmod(big_mod_small(&Ql[l], c->q[l]), c->q[l]);
  }
  double logq = 0.0;
  for (u32 l = 0; l < L; l++) logq += log2((double)c->q[l]);
  double worst = 0.0;
  for (u32 kk = 0; kk < n; kk++) {
    big_t X;
    big_zero(&X);
    for (u32 l = 0; l < L; l++) {
      big_t term = Ql[l];
      big_mul_small(&term, mulmod(x[(u64)l * n + kk], yinv[l], c->q[l]));
      big_add(&X, &term);
    }
    while (big_cmp(&X, &Q) >= 0) big_sub(&X, &Q);
    /* residual v = t*x mod q, centred: distance to the nearest multiple of q */
    big_t v = X;
    big_mul_small(&v, c->t);
    while (big_cmp(&v, &Q) >= 0) big_sub(&v, &Q);
    big_t w = Q;
    big_sub(&w, &v);
    const big_t* m = big_cmp(&v, &w) <= 0 ? &v : &w;
    double mag = 0.0;
    for (int i = BW - 1; i >= 0; i--) mag = mag * 4294967296.0 + (double)m->w[i];
    if (mag > worst) worst = mag;
  }
  free(x); free(sl); free(cs);
  double noise_bits = worst > 0 ? log2(worst / (double)c->t) : 0.0;
  return logq - log2(2.0 * c->t) - noise_bits;
}

#ifdef _OPENMP
#include <omp.h>
int or_num_threads(void) { return omp_get_max_threads(); }
void or_set_threads(int k) { if (k > 0) omp_set_num_threads(k); }
#else
int or_num_threads(void) { return 1; }
void or_set_threads(int k) { (void)k; }
#endif

/* ------------------------------------------------------------------------- */
/* Server-side variant (HE-HDC-SR, Sec. 3): the client encrypts its queries    */
/* ------------------------------------------------------------------------- */
/* Query plaintext (g, i) encrypted with the secret key: c1 = a (domain 6),
 * c0 = -a s + e (domain 7) + Delta m, obj = g*P + i.  ctq: [G][P][2][L][n]. */
void or_encrypt_queries(const or_ctx* c, u64 seed, const int8_t* H, i32 B, const i32* s,
                        u32* ctq) {
  u32 n = c->n, L = c->L;
  u32 G = (u32)((B + c->cap - 1) / c->cap);
#pragma omp parallel
  {
    u32* slots = (u32*)malloc(sizeof(u32) * n);
    u32* m = (u32*)malloc(sizeof(u32) * n);
    u32* a = (u32*)malloc(sizeof(u32) * L * n);
    i32* e = (i32*)malloc(sizeof(i32) * n);
    u32* sl = (u32*)malloc(sizeof(u32) * n);
    u32* as = (u32*)malloc(sizeof(u32) * n);
#pragma omp for schedule(dynamic)
    for (i64 gi = 0; gi < (i64)G * c->P; gi++) {
      u32 g = (u32)(gi / c->P), i = (u32)(gi % c->P);
      query_slots(c, H, B, g, i, slots);
      or_slot_encode(n, c->t, c->zeta, slots, m);
      or_sample_uniform(seed, 6, (u64)gi, n, L, c->q, a);
      or_sample_gauss(seed, 7, (u64)gi, n, c->cdt, e);
      for (u32 l = 0; l < L; l++) {
        u32 p = c->q[l];
        for (u32 kk = 0; kk < n; kk++) sl[kk] = smod(s[kk], p);
        or_polymul(n, p, c->psi[l], a + (u64)l * n, sl, as);
        u32* c0 = ctq + (((u64)gi * 2 + 0) * L + l) * n;
        u32* c1 = ctq + (((u64)gi * 2 + 1) * L + l) * n;
        for (u32 kk = 0; kk < n; kk++) {
          u32 v = submod(smod(e[kk], p), as[kk], p);
          c0[kk] = addmod(v, scaled_msg(c, l, m[kk]), p);
          c1[kk] = a[(u64)l * n + kk];
        }
      }
    }
    free(slots); free(m); free(a); free(e); free(sl); free(as);
  }
}

/* Model plaintexts of the server-side variant: mm[jp][i] = encode(class slots of
 * ciphertext (i, jp)) mod t, coefficient domain.  mm: [Kp][P][n]. */
void or_encode_model_plain(const or_ctx* c, const int8_t* classes, u32* mm) {
  u32 n = c->n;
#pragma omp parallel
  {
    u32* slots = (u32*)malloc(sizeof(u32) * n);
#pragma omp for schedule(dynamic)
    for (i64 ji = 0; ji < (i64)c->Kp * c->P; ji++) {
      u32 jp = (u32)(ji / c->P), i = (u32)(ji % c->P);
      class_slots(c, classes, i, jp, slots);
      or_slot_encode(n, c->t, c->zeta, slots, mm + (u64)ji * n);
    }
    free(slots);
  }
}

/* Server computation: acc[g][jp][poly][l] = sum_i ctq[g][i][poly][l] * lift(mm[jp][i]). */
void or_ctpt_mac(const or_ctx* c, const u32* ctq, i32 B, const u32* mm, u32* acc) {
  u32 n = c->n, L = c->L;
  u32 G = (u32)((B + c->cap - 1) / c->cap);
  i64 jobs = (i64)G * c->Kp * 2 * L;
#pragma omp parallel
  {
    u32* lm = (u32*)malloc(sizeof(u32) * n);
    u32* prod = (u32*)malloc(sizeof(u32) * n);
#pragma omp for schedule(dynamic)
    for (i64 job = 0; job < jobs; job++) {
      u32 l = (u32)(job % L);
      u32 poly = (u32)((job / L) % 2);
      u32 jp = (u32)((job / (2 * L)) % c->Kp);
      u32 g = (u32)(job / (2 * L * c->Kp));
      u32 p = c->q[l];
      u32* out = acc + ((((u64)g * c->Kp + jp) * 2 + poly) * L + l) * n;
      for (u32 kk = 0; kk < n; kk++) out[kk] = 0;
      for (u32 i = 0; i < c->P; i++) {
        const u32* mi = mm + ((u64)jp * c->P + i) * n;
        for (u32 kk = 0; kk < n; kk++) lm[kk] = lift(mi[kk], c->t, p);
        const u32* ct = ctq + ((((u64)g * c->P + i) * 2 + poly) * L + l) * n;
        or_polymul(n, p, c->psi[l], ct, lm, prod);
        for (u32 kk = 0; kk < n; kk++) out[kk] = addmod(out[kk], prod[kk], p);
        if (c->scale_shift && (i + 1) % c->scale_group == 0) {
          u32 u = lift(c->scale_u, c->t, p);  /* scaling operation, as on the client side */
          for (u32 kk = 0; kk < n; kk++) out[kk] = mulmod(out[kk], u, p);
        }
      }
    }
    free(lm); free(prod);
  }
}
