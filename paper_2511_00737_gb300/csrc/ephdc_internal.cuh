// Internal definitions of the EP-HDC CUDA library (sm_103a).
//
// Everything on the path is exact integer arithmetic: residues modulo 30-bit RNS
// primes q_l = 1 (mod 2n) and modulo t = 65537.  Modular products with a fixed
// operand (twiddles, key material) use Shoup's precomputed quotient; products of
// two variable residues accumulate lazily in 64 bits and are reduced once.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ephdc.h"

#define EPHDC_MAXL 8
#define EPHDC_T_DEFAULT 65537u
#define EPHDC_CDT_LEN 38
#define EPHDC_BIGW 10  // words of the multi-word integers used by decryption

// One NTT modulus and its tables (device pointers).
struct ModP {
  uint32_t p;
  uint32_t ninv, ninv_sh;  // n^-1 mod p and its Shoup quotient
  uint64_t mu;             // floor(2^64 / p) for Barrett reduction of 64-bit sums
  const uint2* tw;         // tw[k]  = (psi^brv(k),  Shoup quotient), k in [1, n)
  const uint2* itw;        // itw[k] = (psi^-brv(k), Shoup quotient)
  // the same twiddles for the contiguous pass (the last 5 forward stages, the first 5
  // inverse stages) transposed so that a warp's loads are coalesced:
  // twl[(2^r - 1 + u) * (n/32) + blk] = tw[(n/32 + blk) * 2^r + u], r < 5, u < 2^r
  const uint2* twl;
  const uint2* itwl;
};

// Parameters and tables as seen by kernels (passed by value).
struct DevCtx {
  uint32_t n, logn, L, k, k_in, Kp, r, logr, W, cap_row, cap, P, D, F, bits;
  int32_t shift;
  ModP mq[EPHDC_MAXL];  // the RNS primes
  ModP mt;              // t = 65537
  uint32_t delta[EPHDC_MAXL];  // floor(Q / t) mod q_l
  uint32_t qhat_inv[EPHDC_MAXL];  // (Q / q_l)^-1 mod q_l
  uint32_t big_Q[EPHDC_BIGW];     // Q = prod q_l (little-endian 32-bit words)
  uint32_t big_Qhalf[EPHDC_BIGW]; // floor(Q / 2)
  uint32_t big_Qhat[EPHDC_MAXL][EPHDC_BIGW];  // Q / q_l
  const uint32_t* pos2slot;  // device NTT position j -> slot index rho*(n/2) + col
  const uint32_t* slot2pos;  // slot index -> device NTT position
  const uint32_t* galois;    // galois[j] = 3^(W*2^j) mod 2n, j < logr
  const uint32_t* scatter;   // [(qidx * r + ch) * k_in + jin] -> padded index of the
                             // device position (padi of it, for the slot buffer)
  const uint32_t* hslot;     // [b] = (int8 b mod t) * n^-1 mod t: the packed slot value,
                             // scaled for an inverse transform without the n^-1 step
  uint32_t pack_rows;        // r when query rows pack by vector loads, else 0
  // context scratch used by kernels: fp16 copies of the HDC operands, status word
  uint16_t* xh;              // [max_batch][F] fp16 features
  uint16_t* wh;              // [D][F] fp16 projection
  uint32_t* status;          // nonzero when a bounded device wait gave up
  int32_t ntt_plan;          // pass schedule of the encoding transforms (NttPlan V)
  int32_t hdc_mode;          // HDC projection: 0 persistent GEMM with 128 x 256 tiles and
                             // a 3-stage ring, 1 one 128 x 128 tile per CTA, 2 persistent
                             // with 128 x 128 tiles, 3 as 0 with a 4-stage ring
  uint64_t cdt[EPHDC_CDT_LEN];
  uint32_t t;                // plaintext modulus (prime = 1 mod 2n, < 2^30)
  uint32_t rt;               // Q mod t
  // scaling operation: plaintext i is multiplied by scale_w[l]^(P/g - i/g) mod q_l,
  // scale_w[l] = the centred lift of (2^s)^-1 mod t; scale_g = g (0 = off)
  uint32_t scale_g;
  uint32_t scale_w[EPHDC_MAXL];
  // NTT-domain storage of plaintexts and model: 0 = plaintexts [G][P][L][n] and model
  // [P][O][L][n] (O = 2 k/k_in outputs o = j' * 2 + poly); 1 = coefficient-blocked,
  // [L][n/4][G][P][4] and [L][n/4][P][O][4], so that the 4 coefficients of a block of
  // every (group, plaintext) and (plaintext, output) pair are 16 contiguous bytes and a
  // block's pairs are contiguous (read by the tensor-core multiply-accumulate)
  uint32_t layout;
  // compact model (Sec. 4.1, the model shipped once): only c0 is stored, [P][O/2][L][n],
  // and c1 at device position k of limb l is word64(l n + k) mod q_l of the ChaCha20
  // stream (model_seed, domain 8, ciphertext number), regenerated by the tiled
  // multiply-accumulate as it reads the model
  uint32_t compact;
  uint64_t model_seed;
  // digit model: the model is stored as the tensor-core operand of its signed base-256
  // digits, fp16 tiles [L][n/8][P16][8][R x 16] (P16 = ceil(P/16); R = mdig_rows(Kp):
  // 64 rows when k/k_in <= 8, else 128; tile (l, x/8, i/16, x%8) holds rows
  // r = 4 o + v, columns i%16, at mdig_off(r, i%16); rows o >= O and plaintexts
  // i >= P are zero), read by the digit-outer-product multiply-accumulate
  uint32_t mdig;
};

// byte offset of element (row r, column k) of a 16-column fp16 operand tile in the
// K-major layout without swizzle that tcgen05 descriptors with LBO = 128 and SBO = 256
// describe: 8 x 8 core matrices of 128 bytes, the two column halves 128 bytes apart,
// consecutive 8-row groups 256 bytes apart
__host__ __device__ __forceinline__ uint32_t mdig_off(uint32_t r, uint32_t k) {
  return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
// rows of a digit-model tile: 16 outputs x 4 digits (k/k_in <= 8, an M = 64 operand)
// or 32 outputs x 4 digits (M = 128)
__host__ __device__ __forceinline__ uint32_t mdig_rows(uint32_t Kp) {
  return 2 * Kp <= 16 ? 64u : 128u;
}
// bytes of the digit model
__host__ __device__ __forceinline__ size_t mdig_bytes(uint32_t n, uint32_t L, uint32_t P,
                                                      uint32_t Kp) {
  return (size_t)L * n * ((P + 15) / 16) * mdig_rows(Kp) * 32;
}
// fp16 word index of digit v of model residue (plaintext i, output o, limb l,
// coefficient x) in the digit model with R rows per tile (row 4 o + v: the 4 digits of
// an output sit in 4 consecutive accumulator lanes of one warp)
__host__ __device__ __forceinline__ size_t mdig_index(uint32_t n, uint32_t P, uint32_t R,
                                                      uint32_t i, uint32_t o, uint32_t v,
                                                      uint32_t l, uint32_t x) {
  const uint32_t P16 = (P + 15) / 16;
  const size_t tile = (((size_t)l * (n >> 3) + (x >> 3)) * P16 + (i >> 4)) * 8 + (x & 7);
  return tile * (R * 16) + mdig_off(4 * o + v, i & 15) / 2;
}

// word index of coefficient k of limb l of pair (a, b) in the blocked layout
// [L][n/4][A][B][4] (plaintexts: a = group, b = plaintext; model: a = plaintext,
// b = output)
__host__ __device__ __forceinline__ size_t blk_index(uint32_t n, uint32_t A, uint32_t B,
                                                      uint32_t a, uint32_t b, uint32_t l,
                                                      uint32_t k) {
  return ((((size_t)l * (n >> 2) + (k >> 2)) * A + a) * B + b) * 4 + (k & 3);
}


// ------------------------------------------------------------------ arithmetic
__device__ __forceinline__ uint32_t mulshoup(uint32_t x, uint32_t w, uint32_t wsh, uint32_t p) {
  // x * w mod p in [0, 2p) for any x < 2^32, w < p, wsh = floor(w 2^32 / p)
  return x * w - __umulhi(x, wsh) * p;
}
__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t p) { return x >= p ? x - p : x; }
__device__ __forceinline__ uint32_t addm(uint32_t a, uint32_t b, uint32_t p) {
  return csub(a + b, p);
}
__device__ __forceinline__ uint32_t subm(uint32_t a, uint32_t b, uint32_t p) {
  return a >= b ? a - b : a + p - b;
}
// x mod p for any 64-bit x (Barrett with mu = floor(2^64/p)); result in [0, p)
__device__ __forceinline__ uint32_t red64(uint64_t x, uint32_t p, uint64_t mu) {
  uint64_t qh = __umul64hi(x, mu);
  uint32_t r = (uint32_t)(x - qh * p);  // < 3p < 2^32
  r = csub(r, 2 * p);
  return csub(r, p);
}
__device__ __forceinline__ uint32_t mulm(uint32_t a, uint32_t b, const ModP& m) {
  return red64((uint64_t)a * b, m.p, m.mu);
}

// scale_w[l]^e mod q_l (square and multiply; e is at most P)
__device__ __forceinline__ uint32_t scale_factor(const DevCtx& c, uint32_t l, uint32_t e) {
  const uint32_t p = c.mq[l].p;
  const uint64_t mu = c.mq[l].mu;
  uint32_t r = 1, b = c.scale_w[l];
  while (e) {
    if (e & 1) r = red64((uint64_t)r * b, p, mu);
    b = red64((uint64_t)b * b, p, mu);
    e >>= 1;
  }
  return r;
}

// The scaled message of encryption, round(Q m / t) (ties up) for m in [0, t), reduced
// mod q_l.  Q m = (floor(Q/t) t + (Q mod t)) m, so it is floor(Q/t) m + fix with
// fix = floor(((Q mod t) m + floor((t+1)/2)) / t) < t; the quotient comes from the
// Barrett constant of t and one correction step.
// (The context is read by value: a reference into the kernel-parameter arrays with a
// runtime index would make the compiler copy the whole parameter block to local
// memory.)
struct ScaledMsg {
  uint32_t rt, t, half, dl, p;
  uint64_t tmu, pmu;
  __device__ __forceinline__ ScaledMsg(const DevCtx& c, uint32_t l)
      : rt(c.rt), t(c.t), half((c.t + 1) / 2), dl(c.delta[l]), p(c.mq[l].p), tmu(c.mt.mu),
        pmu(c.mq[l].mu) {}
  __device__ __forceinline__ uint32_t operator()(uint32_t m) const {
    const uint64_t num = (uint64_t)rt * m + half;
    uint64_t fix = __umul64hi(num, tmu);
    if (num - fix * t >= t) fix++;
    return addm(red64((uint64_t)dl * m, p, pmu), red64(fix, p, pmu), p);
  }
};

// shared-memory index with one pad word per 32 (bank-conflict-free NTT passes)
__device__ __forceinline__ uint32_t padi(uint32_t i) { return i + (i >> 5); }
__host__ __device__ constexpr uint32_t padded_words(uint32_t n) { return n + (n >> 5); }

__device__ __forceinline__ uint32_t brev(uint32_t v, uint32_t bits) {
  return __brev(v) >> (32 - bits);
}

// ------------------------------------------------------------------ NTT
// Device NTT order: position j holds a(psi^(2 brv(j) + 1)).  The forward transform
// is the merged negacyclic Cooley-Tukey network (natural order in, bit-reversed
// out); the inverse is the Gentleman-Sande mirror.  Stages are grouped into passes
// of K radix-2 stages held in registers; a thread owns 2^K elements with stride
// S = n / (m0 2^K), where m0 is the block count at the pass's first stage.  The
// last pass uses K = 5 with contiguous elements, so every earlier pass has S >= 32
// and, with one pad word per 32, every pass is bank-conflict-free.
//
// Forward butterflies keep values in [0, 4p) (Harvey); the inverse keeps [0, 2p).

template <int K>
__device__ __forceinline__ void fwd_pass(uint32_t* s, uint32_t logn, uint32_t logm0,
                                         const uint2* __restrict__ tw, uint32_t p) {
  const uint32_t logS = logn - logm0 - K;
  const uint32_t S = 1u << logS;
  const uint32_t groups = 1u << (logn - K);
  const uint32_t m0 = 1u << logm0;
  const uint32_t two_p = 2 * p;
  for (uint32_t gi = threadIdx.x; gi < groups; gi += blockDim.x) {
    const uint32_t blk = gi >> logS, j0 = gi & (S - 1);
    const uint32_t base = (blk << (logS + K)) + j0;
    uint32_t x[1 << K];
#pragma unroll
    for (int e = 0; e < (1 << K); e++) x[e] = s[padi(base + (e << logS))];
#pragma unroll
    for (int r = 0; r < K; r++) {
      const int half = 1 << (K - 1 - r);
      uint2 w[1 << (K - 1)];
#pragma unroll
      for (int u = 0; u < (1 << r); u++) w[u] = __ldg(&tw[((m0 + blk) << r) + u]);
#pragma unroll
      for (int e = 0; e < (1 << K); e++) {
        if (e & half) continue;
        const uint2 ww = w[e >> (K - r)];
        uint32_t X = x[e];
        X = X >= two_p ? X - two_p : X;
        const uint32_t T = mulshoup(x[e + half], ww.x, ww.y, p);
        x[e] = X + T;
        x[e + half] = X - T + two_p;
      }
    }
#pragma unroll
    for (int e = 0; e < (1 << K); e++) s[padi(base + (e << logS))] = x[e];
  }
}

template <int K>
__device__ __forceinline__ void inv_pass(uint32_t* s, uint32_t logn, uint32_t logm0,
                                         const uint2* __restrict__ itw, uint32_t p) {
  const uint32_t logS = logn - logm0 - K;
  const uint32_t S = 1u << logS;
  const uint32_t groups = 1u << (logn - K);
  const uint32_t m0 = 1u << logm0;
  const uint32_t two_p = 2 * p;
  for (uint32_t gi = threadIdx.x; gi < groups; gi += blockDim.x) {
    const uint32_t blk = gi >> logS, j0 = gi & (S - 1);
    const uint32_t base = (blk << (logS + K)) + j0;
    uint32_t x[1 << K];
#pragma unroll
    for (int e = 0; e < (1 << K); e++) x[e] = s[padi(base + (e << logS))];
#pragma unroll
    for (int r = K - 1; r >= 0; r--) {
      const int half = 1 << (K - 1 - r);
      uint2 w[1 << (K - 1)];
#pragma unroll
      for (int u = 0; u < (1 << r); u++) w[u] = __ldg(&itw[((m0 + blk) << r) + u]);
#pragma unroll
      for (int e = 0; e < (1 << K); e++) {
        if (e & half) continue;
        const uint2 ww = w[e >> (K - r)];
        const uint32_t X = x[e], Y = x[e + half];
        uint32_t U = X + Y;
        U = U >= two_p ? U - two_p : U;
        x[e] = U;
        x[e + half] = mulshoup(X - Y + two_p, ww.x, ww.y, p);
      }
    }
#pragma unroll
    for (int e = 0; e < (1 << K); e++) s[padi(base + (e << logS))] = x[e];
  }
}

// pass schedule: the last pass has min(5, logn) stages, the earlier ones <= 5
__device__ __forceinline__ int pass_k(uint32_t logn, int idx, int* npass) {
  const int last = logn < 5 ? (int)logn : 5;
  const int rest = (int)logn - last;
  const int front = (rest + 4) / 5;  // passes before the last
  *npass = front + 1;
  if (idx == front) return last;
  // spread `rest` stages over `front` passes, larger ones first
  const int base = front ? rest / front : 0, extra = front ? rest % front : 0;
  return base + (idx < extra ? 1 : 0);
}

// forward NTT in shared memory (padded layout); input in [0, 4p), output in [0, p)
static __device__ __noinline__ void ntt_fwd_smem(uint32_t* s, uint32_t logn, const ModP m) {
  int np;
  pass_k(logn, 0, &np);
  uint32_t logm0 = 0;
  for (int i = 0; i < np; i++) {
    int K = pass_k(logn, i, &np);
    switch (K) {
      case 1: fwd_pass<1>(s, logn, logm0, m.tw, m.p); break;
      case 2: fwd_pass<2>(s, logn, logm0, m.tw, m.p); break;
      case 3: fwd_pass<3>(s, logn, logm0, m.tw, m.p); break;
      case 4: fwd_pass<4>(s, logn, logm0, m.tw, m.p); break;
      default: fwd_pass<5>(s, logn, logm0, m.tw, m.p); break;
    }
    logm0 += K;
    __syncthreads();
  }
  const uint32_t n = 1u << logn;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    uint32_t v = s[padi(i)];
    v = csub(v, 2 * m.p);
    s[padi(i)] = csub(v, m.p);
  }
  __syncthreads();
}

// inverse NTT in shared memory; input in [0, 2p), output in [0, p)
static __device__ __noinline__ void ntt_inv_smem(uint32_t* s, uint32_t logn, const ModP m) {
  int np;
  pass_k(logn, 0, &np);
  uint32_t logm0 = logn;
  for (int i = np - 1; i >= 0; i--) {
    int K = pass_k(logn, i, &np);
    logm0 -= K;
    switch (K) {
      case 1: inv_pass<1>(s, logn, logm0, m.itw, m.p); break;
      case 2: inv_pass<2>(s, logn, logm0, m.itw, m.p); break;
      case 3: inv_pass<3>(s, logn, logm0, m.itw, m.p); break;
      case 4: inv_pass<4>(s, logn, logm0, m.itw, m.p); break;
      default: inv_pass<5>(s, logn, logm0, m.itw, m.p); break;
    }
    __syncthreads();
  }
  const uint32_t n = 1u << logn;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    uint32_t v = mulshoup(s[padi(i)], m.ninv, m.ninv_sh, m.p);
    s[padi(i)] = csub(v, m.p);
  }
  __syncthreads();
}

// ------------------------------------------------------------------ NTT, compile-time size
// The same networks with log2(n) known at compile time: every stride, pass boundary
// and shared-memory offset is a constant, each element costs one shared load and one
// shared store per pass, and the final reduction (forward) or n^-1 scaling (inverse)
// is folded into the last pass.
// Pass schedules (the "radix" choice): the last pass always has K = min(5, log n)
// contiguous elements; the other log n - 5 stages are split into passes of at most 5
// stages.  V = 0: balanced split; V = 1: radix-32 passes first; V = 2: radix-32
// passes last.  Every split keeps the non-contiguous strides >= 32.
template <int LOGN, int V = 0>
struct NttPlan {
  static constexpr int LAST = LOGN < 5 ? LOGN : 5;
  static constexpr int REST = LOGN - LAST;
  static constexpr int FRONT = (REST + 4) / 5;
  static constexpr int NP = FRONT + 1;
  __host__ __device__ static constexpr int K(int i) {
    return i == FRONT ? LAST
         : V == 1     ? (i < REST / 5 ? 5 : REST - 5 * (REST / 5))
         : V == 2     ? (i == 0 && REST % 5 ? REST % 5 : 5)
                      : (REST / FRONT + (i < REST % FRONT ? 1 : 0));
  }
  __host__ __device__ static constexpr int LOGM0(int i) {
    int s = 0;
    for (int j = 0; j < i; j++) s += K(j);
    return s;
  }
};

// Shared-memory element access (padded layout); the first pass of a transform may
// take a custom loader and the last pass a custom storer, so that the producer
// (slot gather, lift) and the consumer (global store) fuse into the passes.
// A loader or storer that also takes the padded index directly (`at`) lets a pass form
// each element's address as one padded base plus a compile-time offset.
struct SmemLd {
  static constexpr bool kPadded = true;
  const uint32_t* s;
  __device__ __forceinline__ uint32_t operator()(uint32_t i) const { return s[padi(i)]; }
  __device__ __forceinline__ uint32_t at(uint32_t pi) const { return s[pi]; }
};
struct SmemSt {
  static constexpr bool kPadded = true;
  uint32_t* s;
  __device__ __forceinline__ void operator()(uint32_t i, uint32_t v) const { s[padi(i)] = v; }
  __device__ __forceinline__ void at(uint32_t pi, uint32_t v) const { s[pi] = v; }
};
template <class F, class = void>
struct PaddedAccess {
  static constexpr bool value = false;
};
template <class F>
struct PaddedAccess<F, decltype((void)F::kPadded)> {
  static constexpr bool value = F::kPadded;
};

// FINAL: forward -> reduce outputs to [0, p); inverse -> multiply by n^-1, reduce
// NSCALE = false: the inverse's final pass only reduces (its input was scaled by n^-1)
// FERMAT (inverse mod t = 2^16 + 1 only): values stay in [0, t) and the twiddle
// product d w (d <= 2^16, w < 2^16: below 2^32) is reduced without a multiply, as
// 2^16 = -1 (mod t) gives d w = lo + 2^16 hi = lo - hi (mod t)
template <int LOGN, int K, int LOGM0, bool FWD, bool FINAL, class LD, class ST,
          bool NSCALE = true, bool FERMAT = false>
__device__ __forceinline__ void pass_t(const uint2* __restrict__ tw, const ModP& m, LD ld, ST st) {
  constexpr int LOGS = LOGN - LOGM0 - K;
  constexpr uint32_t S = 1u << LOGS;
  static_assert(S == 1 || S >= 32, "pass stride must be contiguous or >= 32");
  constexpr uint32_t GROUPS = 1u << (LOGN - K);
  constexpr uint32_t M0 = 1u << LOGM0;
  // the contiguous pass of a full-size transform reads the transposed twiddle copy
  constexpr bool CONTIG = S == 1 && K == 5;
  const uint32_t p = m.p, two_p = 2 * p;
  const uint2* twl = FWD ? m.twl : m.itwl;
  // (this loop form, a signed iteration count with an exit test and one stage loop for
  // both directions, compiles to fewer live registers than a strided group index)
  for (int itx = 0; itx < (1 << 30); itx++) {
    const uint32_t gi = threadIdx.x + itx * blockDim.x;
    if (gi >= GROUPS) break;
    const uint32_t blk = gi >> LOGS, j0 = gi & (S - 1);
    const uint32_t base = (blk << (LOGS + K)) + j0;
    auto twa = [&](int r, int u) -> const uint2* {
      return CONTIG ? &twl[((1u << r) - 1 + u) * M0 + blk] : &tw[((M0 + blk) << r) + u];
    };
    uint32_t x[1 << K];
    // padded index of element e = padi(base) + e PS, exactly: a contiguous pass has a
    // 32-aligned base, a strided one adds multiples of 32
    constexpr uint32_t PS = S == 1 ? 1 : S + S / 32;
    if constexpr (PaddedAccess<LD>::value) {
      const uint32_t pb = padi(base);
#pragma unroll
      for (int e = 0; e < (1 << K); e++) x[e] = ld.at(pb + e * PS);
    } else {
#pragma unroll
      for (int e = 0; e < (1 << K); e++) x[e] = ld(base + e * S);
    }
#pragma unroll
    for (int rr = 0; rr < K; rr++) {
      const int r = FWD ? rr : K - 1 - rr;
      const int half = 1 << (K - 1 - r);
      uint2 w[1 << (K - 1)];
#pragma unroll
      for (int u = 0; u < (1 << r); u++) w[u] = __ldg(twa(r, u));
#pragma unroll
      for (int e = 0; e < (1 << K); e++) {
        if (e & half) continue;
        const uint2 ww = w[e >> (K - r)];
        if (FWD) {
          const uint32_t X = min(x[e], x[e] - two_p);
          const uint32_t T = mulshoup(x[e + half], ww.x, ww.y, p);
          x[e] = X + T;
          x[e + half] = X - T + two_p;
        } else if (FERMAT) {
          const uint32_t X = x[e], Y = x[e + half];
          const uint32_t U = X + Y, D0 = X - Y + p;  // p = t here; both in [0, 2t)
          x[e] = min(U, U - p);
          const uint32_t D = min(D0, D0 - p);        // [0, t)
          const uint32_t P = D * ww.x;               // < 2^16 (2^16 - 1) < 2^32
          const uint32_t R = (P & 0xFFFFu) + p - (P >> 16);  // [1, 2t)
          x[e + half] = min(R, R - p);
        } else {
          const uint32_t X = x[e], Y = x[e + half];
          const uint32_t U = X + Y;
          x[e] = min(U, U - two_p);
          x[e + half] = mulshoup(X - Y + two_p, ww.x, ww.y, p);
        }
      }
    }
    if (FINAL) {
#pragma unroll
      for (int e = 0; e < (1 << K); e++) {
        if (FWD) {
          const uint32_t v = min(x[e], x[e] - two_p);
          x[e] = min(v, v - p);
        } else if (NSCALE) {
          const uint32_t v = mulshoup(x[e], m.ninv, m.ninv_sh, p);
          x[e] = min(v, v - p);
        } else {
          x[e] = min(x[e], x[e] - p);
        }
      }
    }
    if constexpr (PaddedAccess<ST>::value) {
      const uint32_t pb = padi(base);
#pragma unroll
      for (int e = 0; e < (1 << K); e++) st.at(pb + e * PS, x[e]);
    } else {
#pragma unroll
      for (int e = 0; e < (1 << K); e++) st(base + e * S, x[e]);
    }
  }
}

template <int LOGN, int I, class LD, class ST, int V = 0>
__device__ __forceinline__ void fwd_passes(uint32_t* s, const ModP& m, LD ld, ST st) {
  using Pl = NttPlan<LOGN, V>;
  if constexpr (I < Pl::NP) {
    constexpr bool first = I == 0, last = I == Pl::NP - 1;
    if constexpr (first && last) {
      pass_t<LOGN, Pl::K(I), Pl::LOGM0(I), true, true>(m.tw, m, ld, st);
    } else if constexpr (first) {
      pass_t<LOGN, Pl::K(I), Pl::LOGM0(I), true, false>(m.tw, m, ld, SmemSt{s});
    } else if constexpr (last) {
      pass_t<LOGN, Pl::K(I), Pl::LOGM0(I), true, true>(m.tw, m, SmemLd{s}, st);
    } else {
      pass_t<LOGN, Pl::K(I), Pl::LOGM0(I), true, false>(m.tw, m, SmemLd{s}, SmemSt{s});
    }
    __syncthreads();
    fwd_passes<LOGN, I + 1, LD, ST, V>(s, m, ld, st);
  }
}
template <int LOGN, int I, class LD, class ST, int V = 0, bool NSCALE = true,
          bool FERMAT = false>
__device__ __forceinline__ void inv_passes(uint32_t* s, const ModP& m, LD ld, ST st) {
  using Pl = NttPlan<LOGN, V>;
  if constexpr (I >= 0) {
    constexpr bool first = I == Pl::NP - 1, last = I == 0;
    if constexpr (first && last) {
      pass_t<LOGN, Pl::K(I), Pl::LOGM0(I), false, true, LD, ST, NSCALE, FERMAT>(m.itw, m, ld,
                                                                                 st);
    } else if constexpr (first) {
      pass_t<LOGN, Pl::K(I), Pl::LOGM0(I), false, false, LD, SmemSt, true, FERMAT>(
          m.itw, m, ld, SmemSt{s});
    } else if constexpr (last) {
      pass_t<LOGN, Pl::K(I), Pl::LOGM0(I), false, true, SmemLd, ST, NSCALE, FERMAT>(
          m.itw, m, SmemLd{s}, st);
    } else {
      pass_t<LOGN, Pl::K(I), Pl::LOGM0(I), false, false, SmemLd, SmemSt, true, FERMAT>(
          m.itw, m, SmemLd{s}, SmemSt{s});
    }
    __syncthreads();
    inv_passes<LOGN, I - 1, LD, ST, V, NSCALE, FERMAT>(s, m, ld, st);
  }
}
// Forward NTT: `ld(i)` supplies natural-order input i (values in [0, 4p)) to the first
// pass, `st(j, v)` receives device-order output j (in [0, p)) from the last pass;
// shared buffer `s` (padded) carries the passes in between.  Ends with a barrier.
template <int LOGN, class LD, class ST, int V = 0>
__device__ __forceinline__ void ntt_fwd_io(uint32_t* s, const ModP& m, LD ld, ST st) {
  fwd_passes<LOGN, 0, LD, ST, V>(s, m, ld, st);
}
// Inverse NTT: device-order input (values in [0, 2p)) in, natural-order output in
// [0, p) out.  Ends with a barrier.
template <int LOGN, class LD, class ST, int V = 0, bool NSCALE = true, bool FERMAT = false>
__device__ __forceinline__ void ntt_inv_io(uint32_t* s, const ModP& m, LD ld, ST st) {
  inv_passes<LOGN, NttPlan<LOGN, V>::NP - 1, LD, ST, V, NSCALE, FERMAT>(s, m, ld, st);
}
// in-place variants on the padded shared buffer
template <int LOGN, int V = 0>
__device__ __forceinline__ void ntt_fwd_t(uint32_t* s, const ModP& m) {
  ntt_fwd_io<LOGN, SmemLd, SmemSt, V>(s, m, SmemLd{s}, SmemSt{s});
}
template <int LOGN, int V = 0, bool NSCALE = true, bool FERMAT = false>
__device__ __forceinline__ void ntt_inv_t(uint32_t* s, const ModP& m) {
  ntt_inv_io<LOGN, SmemLd, SmemSt, V, NSCALE, FERMAT>(s, m, SmemLd{s}, SmemSt{s});
}

// dispatch a kernel template on log2(n) (n = 1024 .. 16384)
#define EPHDC_DISPATCH_LOGN(logn, LOGN_, ...)            \
  switch (logn) {                                        \
    case 10: { constexpr int LOGN_ = 10; __VA_ARGS__; } break; \
    case 11: { constexpr int LOGN_ = 11; __VA_ARGS__; } break; \
    case 12: { constexpr int LOGN_ = 12; __VA_ARGS__; } break; \
    case 13: { constexpr int LOGN_ = 13; __VA_ARGS__; } break; \
    case 14: { constexpr int LOGN_ = 14; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;               \
  }

// ------------------------------------------------------------------ ChaCha20 (RFC 8439)
__device__ __forceinline__ uint32_t rotl(uint32_t v, int c) { return (v << c) | (v >> (32 - c)); }
#define EPHDC_QR(a, b, c, d)                 \
  a += b; d ^= a; d = rotl(d, 16);           \
  c += d; b ^= c; b = rotl(b, 12);           \
  a += b; d ^= a; d = rotl(d, 8);            \
  c += d; b ^= c; b = rotl(b, 7);

// block `counter` of the stream keyed by seed with nonce (domain, obj_hi, obj_lo)
__device__ __forceinline__ void chacha_block(uint64_t seed, uint32_t domain, uint64_t obj,
                                             uint32_t counter, uint32_t out[16]) {
  const uint32_t in[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u,
                           (uint32_t)seed, (uint32_t)(seed >> 32), 0, 0, 0, 0, 0, 0,
                           counter, domain, (uint32_t)(obj >> 32), (uint32_t)obj};
  uint32_t x0 = in[0], x1 = in[1], x2 = in[2], x3 = in[3], x4 = in[4], x5 = in[5], x6 = in[6],
           x7 = in[7], x8 = in[8], x9 = in[9], x10 = in[10], x11 = in[11], x12 = in[12],
           x13 = in[13], x14 = in[14], x15 = in[15];
#pragma unroll 1
  for (int i = 0; i < 10; i++) {
    EPHDC_QR(x0, x4, x8, x12) EPHDC_QR(x1, x5, x9, x13) EPHDC_QR(x2, x6, x10, x14)
    EPHDC_QR(x3, x7, x11, x15) EPHDC_QR(x0, x5, x10, x15) EPHDC_QR(x1, x6, x11, x12)
    EPHDC_QR(x2, x7, x8, x13) EPHDC_QR(x3, x4, x9, x14)
  }
  out[0] = x0 + in[0]; out[1] = x1 + in[1]; out[2] = x2 + in[2]; out[3] = x3 + in[3];
  out[4] = x4 + in[4]; out[5] = x5 + in[5]; out[6] = x6 + in[6]; out[7] = x7 + in[7];
  out[8] = x8 + in[8]; out[9] = x9 + in[9]; out[10] = x10 + in[10]; out[11] = x11 + in[11];
  out[12] = x12 + in[12]; out[13] = x13 + in[13]; out[14] = x14 + in[14];
  out[15] = x15 + in[15];
}

// ------------------------------------------------------------------ samplers
// Gaussian coefficient from one 64-bit word: -19 + #{m : u >= cdt[m]}
__device__ __forceinline__ int32_t cdt_sample(const DevCtx& c, uint64_t u) {
  int32_t cnt = 0;
#pragma unroll
  for (int m = 0; m < EPHDC_CDT_LEN; m++) cnt += u >= c.cdt[m];
  return cnt - 19;
}

// buf[padi(k)] = uniform coefficient k of limb l: 64-bit word l*n + k mod q_l
__device__ __forceinline__ void fill_uniform(const DevCtx& c, uint64_t seed, uint32_t dom,
                                             uint64_t obj, uint32_t l, uint32_t* buf) {
  const uint32_t p = c.mq[l].p;
  const uint64_t mu = c.mq[l].mu;
  // 8 coefficients (16 words) per ChaCha block; first word64 index l*n is a multiple of 8
  for (uint32_t b = threadIdx.x; b < c.n / 8; b += blockDim.x) {
    uint32_t w[16];
    chacha_block(seed, dom, obj, (uint32_t)(((uint64_t)l * c.n) / 8 + b), w);
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const uint64_t v = (uint64_t)w[2 * u] | ((uint64_t)w[2 * u + 1] << 32);
      buf[padi(b * 8 + u)] = red64(v, p, mu);
    }
  }
}

// buf[padi(k)] = Gaussian coefficient k mod q_l
__device__ __forceinline__ void fill_gauss(const DevCtx& c, uint64_t seed, uint32_t dom,
                                           uint64_t obj, uint32_t p, uint32_t* buf) {
  for (uint32_t b = threadIdx.x; b < c.n / 8; b += blockDim.x) {
    uint32_t w[16];
    chacha_block(seed, dom, obj, b, w);
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const uint64_t v = (uint64_t)w[2 * u] | ((uint64_t)w[2 * u + 1] << 32);
      const int32_t e = cdt_sample(c, v);
      buf[padi(b * 8 + u)] = e < 0 ? (uint32_t)((int32_t)p + e) : (uint32_t)e;
    }
  }
}

// ------------------------------------------------------------------ query slots
// Slot vector of query plaintext (g, i) in device NTT order, values mod t, into the
// zeroed padded buffer mb (Sec. 3, SIMD form): query beta = g*cap + qidx (qidx =
// rho*cap_row + qq) and dimension d = i*r + ch land in slot (rho, ch*W +
// jin*cap_row + qq) for every jin < k_in.  Each value goes to its k_in device
// positions through the context's scatter table (padded indices).  The value written
// is h * n^-1 mod t (table hslot), so the inverse transform that follows skips its
// n^-1 step (ntt_inv_t<..., false>).  No barrier.
//
// Rows path (c.pack_rows = r, with (r, k_in) one of (8, 1), (16, 1), (4, 2): D a
// multiple of r, H aligned to r bytes): a thread takes whole query rows, the row's r
// bytes in one vector load and its r k_in table entries in 16-byte loads, and issues
// the loads of 32 / (r k_in) rows before the first store, so a CTA waits for one
// memory round trip instead of one per row.
// Generic path: threads walk the cap x r block of H byte by byte (consecutive
// threads read consecutive bytes of a query row).
template <int R> struct PackRow;
template <> struct PackRow<4> { using T = uint32_t; };
template <> struct PackRow<8> { using T = uint2; };
template <> struct PackRow<16> { using T = uint4; };

__device__ __forceinline__ uint32_t row_word(uint32_t v, int) { return v; }
__device__ __forceinline__ uint32_t row_word(const uint2& v, int w) { return w ? v.y : v.x; }
__device__ __forceinline__ uint32_t row_word(const uint4& v, int w) {
  return w == 0 ? v.x : w == 1 ? v.y : w == 2 ? v.z : v.w;
}

template <int R, int KIN>
__device__ __forceinline__ void pack_query_rows(const DevCtx& c, const int8_t* __restrict__ H,
                                                uint32_t qlim, uint32_t g, uint32_t i,
                                                uint32_t* mb) {
  using Row = typename PackRow<R>::T;
  constexpr int E = R * KIN;     // table entries per row (a multiple of 4)
  constexpr int QPT = 32 / E;    // rows in flight per thread
  const uint32_t D = c.D;
  const int8_t* Hg = H + (size_t)g * c.cap * D + (size_t)i * R;
  for (uint32_t q0 = threadIdx.x; q0 < qlim; q0 += QPT * blockDim.x) {
    Row hv[QPT];
    uint4 sc[QPT][E / 4];
#pragma unroll
    for (int u = 0; u < QPT; u++) {
      const uint32_t q = q0 + u * blockDim.x;
      if (q < qlim) {
        hv[u] = __ldg(reinterpret_cast<const Row*>(Hg + (size_t)q * D));
        const uint4* st = reinterpret_cast<const uint4*>(c.scatter + (size_t)q * E);
#pragma unroll
        for (int v = 0; v < E / 4; v++) sc[u][v] = __ldg(st + v);
      }
    }
#pragma unroll
    for (int u = 0; u < QPT; u++) {
      if (q0 + u * blockDim.x >= qlim) continue;
#pragma unroll
      for (int e = 0; e < R; e++) {
        const uint32_t b = (row_word(hv[u], e >> 2) >> (8 * (e & 3))) & 0xFFu;
        const uint32_t v = __ldg(&c.hslot[b]);
#pragma unroll
        for (int j = 0; j < KIN; j++) {
          const int x = e * KIN + j;
          mb[row_word(sc[u][x >> 2], x & 3)] = v;
        }
      }
    }
  }
}

__device__ __forceinline__ void pack_query_slots(const DevCtx& c, const int8_t* __restrict__ H,
                                                 int B, uint32_t g, uint32_t i, uint32_t* mb) {
  const uint32_t qlim = min((uint32_t)c.cap, (uint32_t)(B - (int)(g * c.cap)));
  const uint32_t rows = c.pack_rows;
  if (rows && ((uintptr_t)H & (rows - 1)) == 0) {
    if (rows == 8) return pack_query_rows<8, 1>(c, H, qlim, g, i, mb);
    if (rows == 16) return pack_query_rows<16, 1>(c, H, qlim, g, i, mb);
    if (rows == 4) return pack_query_rows<4, 2>(c, H, qlim, g, i, mb);
  }
  const uint32_t d0 = i * c.r;
  const uint32_t r = c.r, logr = c.logr, kin = c.k_in, D = c.D;
  const uint32_t dlim = D - d0 < r ? D - d0 : r;
  const int8_t* Hg = H + (size_t)g * c.cap * D + d0;
  const uint32_t total = qlim << logr;
  for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const uint32_t qidx = idx >> logr, ch = idx & (r - 1);
    if (ch >= dlim) continue;
    const uint32_t v = __ldg(&c.hslot[(uint8_t)Hg[(size_t)qidx * D + ch]]);
    const uint32_t* sc = c.scatter + (size_t)idx * kin;
    for (uint32_t jin = 0; jin < kin; jin++) mb[__ldg(&sc[jin])] = v;
  }
}

// ------------------------------------------------------------------ host context
struct ephdc_ctx_impl;  // defined in host.cu

// launch helpers implemented in the kernel translation units
namespace ephdc {
// X == NULL: the fp16 features are already in c.xh (see launch_gather_widen)
cudaError_t launch_wait_selfcheck(const DevCtx& c, long long limit_cycles, uint32_t code,
                                  cudaStream_t st);
cudaError_t launch_hdc_encode(const DevCtx& c, const int8_t* X, const int8_t* Wt, int B,
                              int8_t* H, cudaStream_t st);
// rows of up to 64 requests, packed back to back into c.xh (fp16)
struct GatherTable {
  const int8_t* ptr[64];
  int32_t off[65];
  int32_t count;
};
cudaError_t launch_gather_widen(const DevCtx& c, const GatherTable& t, cudaStream_t st);
// ni > 0: plaintexts i0 .. i0 + ni - 1 of every group only, into a buffer of ni
// plaintexts per group
cudaError_t launch_encode_plain(const DevCtx& c, const int8_t* H, int B, uint32_t* pt,
                                cudaStream_t st, uint32_t i0 = 0,
                               uint32_t ni = 0);
cudaError_t launch_mac(const DevCtx& c, const uint32_t* pt, int G, const uint32_t* model,
                       uint32_t* partial, int splits, uint32_t* acc, cudaStream_t st);
// acc[x] = sum over splits of partial[split][x] mod q_l, x < words
cudaError_t launch_mac_reduce(const DevCtx& c, const uint32_t* partial, int splits, size_t words,
                              uint32_t* acc, cudaStream_t st);
// tiling of the multi-group MAC: gt groups x ot outputs per warp, gc groups per
// CTA, ic plaintext indices per shared-memory chunk
struct MacTiling {
  int gt, ot, gc, ic;
};
// pP > 0: a chunk of a pass (plaintexts mi0 .. mi0 + cnt - 1 of the model against a
// buffer of pP plaintexts per group), added into acc when accum != 0
cudaError_t launch_mac_tiled(const DevCtx& c, const uint32_t* pt, int G, const uint32_t* model,
                             uint32_t* acc, const MacTiling& t, cudaStream_t st, int pP = 0,
                             int mi0 = 0, int cnt = 0, int accum = 0);
// the same accumulators through the exact byte-split tensor-core product (k/k_in <= 16)
cudaError_t launch_mac_tc(const DevCtx& c, const uint32_t* pt, int G, const uint32_t* model,
                          uint32_t* acc, cudaStream_t st);
cudaError_t launch_mac_uv(const DevCtx& c, const uint32_t* pt, int G, const uint16_t* model,
                          uint32_t* acc, int cluster, cudaStream_t st);
cudaError_t launch_rotate_sum(const DevCtx& c, uint32_t* acc, uint32_t* tmp, uint32_t* digits,
                              int count, const uint32_t* gk, cudaStream_t st);
cudaError_t launch_export(const DevCtx& c, const uint32_t* acc, int count, uint32_t* out,
                          cudaStream_t st);
cudaError_t launch_keygen(const DevCtx& c, uint64_t seed, uint32_t* sk, uint32_t* gk,
                          cudaStream_t st);
cudaError_t launch_encrypt_model(const DevCtx& c, const int8_t* classes, const uint32_t* sk,
                                 uint64_t seed, uint32_t* model, cudaStream_t st);
// server-side variant (HE-HDC-SR): the client encrypts its query plaintexts, the
// server holds the class hypervectors as plaintexts
cudaError_t launch_encrypt_queries(const DevCtx& c, const int8_t* H, int B, const uint32_t* sk,
                                   uint64_t seed, uint32_t* ctq, cudaStream_t st);
cudaError_t launch_encode_model_plain(const DevCtx& c, const int8_t* classes, uint32_t* mm,
                                      cudaStream_t st);
cudaError_t launch_ctpt_mac(const DevCtx& c, const uint32_t* ctq, int G, const uint32_t* mm,
                            uint32_t* partial, int splits_max, uint32_t* acc, cudaStream_t st);
// the noise-growth experiment (findDmax): prefix phases in the coefficient domain,
// decryption of phases already in the coefficient domain, first wrong prefix
int prefix_chunks(const DevCtx& c, int D);
cudaError_t launch_prefix_phases(const DevCtx& c, const uint32_t* pt, const uint32_t* model,
                                 const uint32_t* sk, int D, uint32_t* X, uint32_t* T,
                                 cudaStream_t st);
cudaError_t launch_decrypt_phases(const DevCtx& c, uint32_t* xbuf, int count, int B,
                                  uint32_t* scores, cudaStream_t st);
cudaError_t launch_first_wrong(const DevCtx& c, const int8_t* H, const int8_t* cls, int B, int D,
                               const uint32_t* scores, int* first, cudaStream_t st);
// seeded model message: c0 halves in the coefficient domain, and back with c1 regenerated
cudaError_t launch_model_to_seeded(const DevCtx& c, const uint32_t* model, uint32_t* c0w,
                                  cudaStream_t st);
cudaError_t launch_model_from_seeded(const DevCtx& c, const uint32_t* c0w, uint64_t seed,
                                    uint32_t* model, cudaStream_t st);
cudaError_t launch_decrypt_scores(const DevCtx& c, const uint32_t* sk, const uint32_t* ct,
                                  int B, uint32_t* xbuf, uint32_t* scores, cudaStream_t st);
cudaError_t launch_ntt_natural(const DevCtx& c, uint32_t limb, uint32_t* poly, int count,
                               int inverse, cudaStream_t st);
cudaError_t launch_unblock(const DevCtx& c, const uint32_t* src, uint32_t* dst, uint32_t A,
                           uint32_t B, cudaStream_t st);
cudaError_t launch_expand_compact(const DevCtx& c, const uint32_t* c0, uint32_t* full,
                                  cudaStream_t st);
cudaError_t launch_undigit(const DevCtx& c, const uint16_t* mdig, uint32_t* model,
                           cudaStream_t st);
cudaError_t launch_model_to_digits(const DevCtx& c, const uint32_t* model, uint16_t* mdig,
                                   cudaStream_t st);
cudaError_t launch_to_coeff(const DevCtx& c, const uint32_t* in, uint32_t* out, int count,
                            int limbs_per_item, int in_stride_words, int limb_stride_words,
                            int limb0_is_digit_major, cudaStream_t st);
cudaError_t launch_sk_to_coeff(const DevCtx& c, const uint32_t* sk, int32_t* out, uint32_t* tmp,
                               cudaStream_t st);
// context accessors for entry points defined outside host.cu
const DevCtx* ctx_dev(const ephdc_ctx* c);
int ctx_device(const ephdc_ctx* c);
ephdc_status ctx_fail(ephdc_ctx* c, ephdc_status s, const char* msg);
void ctx_clear_error(ephdc_ctx* c);
}  // namespace ephdc
