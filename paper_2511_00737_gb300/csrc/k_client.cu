// Client-side hot path kernels (Sec. 3, Sec. 4.1):
//   encode_plain  slot packing of query hypervectors + inverse NTT mod t (BFV batch
//                 encoding, EncPt) + centred lift + forward NTT per RNS limb
//   mac           plaintext x ciphertext multiply-accumulate over the plaintexts
//                 (HE compute): streams the NTT-domain encrypted model from HBM
//   rotate_sum    log2(r) Galois rotations with BV key switching, each added back
//   export        inverse NTT of the score ciphertexts to the coefficient domain
// The transforms are instantiated per ring degree (log2 n = 10..14).
#include <cooperative_groups.h>

#include "ephdc_internal.cuh"

namespace cg = cooperative_groups;

namespace {

__device__ __forceinline__ uint32_t galois_pos(uint32_t j, uint32_t g, uint32_t logn) {
  // device position holding exponent e_j * g (mod 2n), e_j = 2 brv(j) + 1
  const uint32_t n2mask = (2u << logn) - 1;
  const uint32_t e = 2 * brev(j, logn) + 1;
  const uint32_t eg = (e * g) & n2mask;
  return brev((eg - 1) >> 1, logn);
}

// ------------------------------------------------------------------ EncPt
// centred lift of a coefficient in [0, t) into Z_{q_l}: v, or v + q_l - t above t/2
struct CentredLift {
  static constexpr bool kPadded = true;
  const uint32_t* s;
  uint32_t thalf, p_minus_t;
  __device__ __forceinline__ uint32_t at(uint32_t pi) const {
    const uint32_t v = s[pi];
    return v <= thalf ? v : v + p_minus_t;
  }
};
// the same lift from the compact copy of the coefficients: the centred value c in
// [-32768, 32768] as int16 (padded index), except c = 32768, which int16 cannot hold:
// stored as 0 with its bit set in `big` (one bit per padded index)
struct CompactLift {
  static constexpr bool kPadded = true;
  const int16_t* s;
  const uint32_t* big;
  uint32_t p;
  __device__ __forceinline__ uint32_t at(uint32_t pi) const {
    const int c = s[pi];
    const uint32_t v = c < 0 ? (uint32_t)(c + (int)p) : (uint32_t)c;
    return (big[pi >> 5] >> (pi & 31)) & 1u ? 32768u : v;
  }
};
// shared memory of the encoder: two padded u32 buffers, or (n = 16384, so that two
// CTAs fit on an SM) one u32 buffer plus the compact coefficient copy
__host__ __device__ constexpr size_t encode_smem_bytes(uint32_t logn) {
  return logn >= 14 ? padded_words(1u << logn) * 4 + padded_words(1u << logn) * 2 +
                          (padded_words(1u << logn) / 32 + 1) * 4
                    : 2 * (size_t)padded_words(1u << logn) * 4;
}

// One CTA per plaintext (g, i).  The query slots are packed (pack_query_slots), the
// inverse NTT mod t gives the plaintext coefficients, and for each limb the centred
// lift feeds the forward NTT, whose output is staged in shared memory and stored
// with 16-byte writes.  (The scaling operation, when on, is a separate pass.)
template <int LOGN, int V>
__global__ void __launch_bounds__(256, LOGN >= 14 ? 2 : 3)
    k_encode_plain(DevCtx c, const int8_t* __restrict__ H, int B, uint32_t* __restrict__ pt,
                   uint32_t i0, uint32_t ni) {
  constexpr uint32_t N = 1u << LOGN;
  constexpr bool CPT = LOGN >= 14;  // compact coefficient copy
  extern __shared__ uint32_t sm[];
  uint32_t* wb = sm;
  // the coefficients mod t: a second u32 buffer, or the compact copy filled from wb
  uint32_t* mb = CPT ? wb : sm + padded_words(N);
  int16_t* m16 = reinterpret_cast<int16_t*>(sm + padded_words(N));
  uint32_t* big = reinterpret_cast<uint32_t*>(m16 + padded_words(N));
  // block gi: plaintext i0 + gi % ni of group gi / ni, stored as plaintext gi of a
  // buffer of ni plaintexts per group (the whole pass: i0 = 0, ni = P)
  const uint32_t gi = blockIdx.x;
  const uint32_t g = gi / ni, i = i0 + (gi - g * ni);
  // with cap r k_in = n, a full group and a full D-chunk write every slot exactly once
  const bool every_slot = c.cap * c.r * c.k_in == N && (g + 1) * c.cap <= (uint32_t)B &&
                          (i + 1) * c.r <= c.D;
  if (!every_slot) {
    for (uint32_t j = threadIdx.x; j < N; j += blockDim.x) mb[padi(j)] = 0;
    __syncthreads();
  }
  pack_query_slots(c, H, B, g, i, mb);
  __syncthreads();
  // slots (scaled by n^-1) -> coefficients in [0, t); t = 2^16 + 1 without multiplies
  // in the reductions
  if (c.t == 65537u) ntt_inv_t<LOGN, V, false, true>(mb, c.mt);
  else ntt_inv_t<LOGN, V, false>(mb, c.mt);
  const uint32_t t = c.t, thalf = (t - 1) / 2;
  if (CPT) {  // wb -> the compact copy (centred values; 32768 flagged)
    for (uint32_t w = threadIdx.x; w < padded_words(N) / 32 + 1; w += blockDim.x) big[w] = 0;
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
      const uint32_t pi = padi(k), v = wb[pi];
      const int cv = v <= thalf ? (int)v : (int)v - (int)t;
      if (cv == 32768) atomicOr(&big[pi >> 5], 1u << (pi & 31));
      m16[pi] = (int16_t)(cv == 32768 ? 0 : cv);
    }
    __syncthreads();
  }
  for (uint32_t l = 0; l < c.L; l++) {
    const ModP m = c.mq[l];
    if constexpr (CPT) {
      ntt_fwd_io<LOGN, CompactLift, SmemSt, V>(wb, m, CompactLift{m16, big, m.p}, SmemSt{wb});
    } else {
      const CentredLift lift{mb, thalf, m.p - t};
      ntt_fwd_io<LOGN, CentredLift, SmemSt, V>(wb, m, lift, SmemSt{wb});
    }
    if (c.layout) {  // coefficient-blocked: 16 bytes per (coefficient block, g, i)
      const uint32_t G = ((uint32_t)B + c.cap - 1) / c.cap;
      uint4* dst = reinterpret_cast<uint4*>(pt);
      for (uint32_t k = threadIdx.x; k < N / 4; k += blockDim.x) {
        const uint32_t* w = wb + padi(4 * k);
        dst[blk_index(N, G, c.P, g, i, l, 4 * k) >> 2] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    } else {
      uint4* dst = reinterpret_cast<uint4*>(pt + ((size_t)gi * c.L + l) * N);
      for (uint32_t k = threadIdx.x; k < N / 4; k += blockDim.x) {
        const uint32_t* w = wb + padi(4 * k);  // the 4 words never straddle a pad word
        dst[k] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    __syncthreads();
  }
}

// Scaling operation folded into the plaintexts (only when it is on): the accumulator
// scaled after every g products equals, mod q_l, the sum of the products with
// plaintext i multiplied by w^(floor(P/g) - floor(i/g)).  One CTA per plaintext.
__global__ void __launch_bounds__(256) k_scale_plain(DevCtx c, uint32_t* __restrict__ pt) {
  const uint32_t gi = blockIdx.x;
  const uint32_t i = gi % c.P, g = gi / c.P, G = gridDim.x / c.P;
  for (uint32_t l = 0; l < c.L; l++) {
    const uint32_t p = c.mq[l].p;
    const uint32_t w = scale_factor(c, l, c.P / c.scale_g - i / c.scale_g);
    const uint32_t wsh = (uint32_t)(((uint64_t)w << 32) / p);
    uint4* q = reinterpret_cast<uint4*>(pt + ((size_t)gi * c.L + l) * c.n);
    for (uint32_t k = threadIdx.x; k < c.n / 4; k += blockDim.x) {
      // 4 coefficients of one block: contiguous in either layout
      uint4* qk = c.layout
                      ? reinterpret_cast<uint4*>(pt) + (blk_index(c.n, G, c.P, g, i, l, 4 * k) >> 2)
                      : q + k;
      uint4 v = *qk;
      v.x = csub(mulshoup(v.x, w, wsh, p), p);
      v.y = csub(mulshoup(v.y, w, wsh, p), p);
      v.z = csub(mulshoup(v.z, w, wsh, p), p);
      v.w = csub(mulshoup(v.w, w, wsh, p), p);
      *qk = v;
    }
  }
}

// ------------------------------------------------------------------ MAC
// partial[split][g][o][l][n] = sum_{i in split} pt[g][i][l] * model[i][o][l]  (mod q_l),
// o = jp*2 + poly.  A thread owns 4 consecutive coefficients of one limb and OC
// outputs; products (< 2^60) accumulate in 64 bits, reduced every 15 terms.
template <int OC>
__global__ void __launch_bounds__(256) k_mac(DevCtx c, const uint32_t* __restrict__ pt,
                                             const uint32_t* __restrict__ model,
                                             uint32_t* __restrict__ partial, int G, int splits,
                                             int o0, int nout) {
  const uint32_t quads = c.n >> 2;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= c.L * quads) return;
  const uint32_t l = tid / quads, quad = tid - l * quads;
  const uint32_t g = blockIdx.y, split = blockIdx.z;
  const uint32_t per = (c.P + splits - 1) / splits;
  const uint32_t i0 = split * per, i1 = min(c.P, i0 + per);
  const uint32_t p = c.mq[l].p;
  const uint64_t mu = c.mq[l].mu;
  const uint32_t O = 2 * c.Kp;
  uint64_t acc[OC][4];
#pragma unroll
  for (int o = 0; o < OC; o++)
#pragma unroll
    for (int e = 0; e < 4; e++) acc[o][e] = 0;
  const uint4* ptp = reinterpret_cast<const uint4*>(pt + (((size_t)g * c.P) * c.L + l) * c.n) + quad;
  const size_t pt_step = (size_t)c.L * quads;  // uint4 per plaintext
  const uint4* mp = reinterpret_cast<const uint4*>(model + (size_t)l * c.n) + quad;
  const size_t out_step = (size_t)c.L * quads;    // uint4 per (ct, poly)
  const size_t i_step = (size_t)O * out_step;      // uint4 per plaintext index
  uint32_t cnt = 0;
  for (uint32_t i = i0; i < i1; i++) {
    const uint4 a = __ldg(ptp + (size_t)i * pt_step);
#pragma unroll
    for (int o = 0; o < OC; o++) {
      if (o < nout) {
        const uint4 b = __ldg(mp + (size_t)i * i_step + (size_t)(o0 + o) * out_step);
        acc[o][0] += (uint64_t)a.x * b.x;
        acc[o][1] += (uint64_t)a.y * b.y;
        acc[o][2] += (uint64_t)a.z * b.z;
        acc[o][3] += (uint64_t)a.w * b.w;
      }
    }
    if (++cnt == 15) {
      cnt = 0;
#pragma unroll
      for (int o = 0; o < OC; o++)
#pragma unroll
        for (int e = 0; e < 4; e++) acc[o][e] = red64(acc[o][e], p, mu);
    }
  }
#pragma unroll
  for (int o = 0; o < OC; o++) {
    if (o < nout) {
      uint4 v = make_uint4(red64(acc[o][0], p, mu), red64(acc[o][1], p, mu),
                           red64(acc[o][2], p, mu), red64(acc[o][3], p, mu));
      uint4* dst = reinterpret_cast<uint4*>(
          partial + ((((size_t)split * G + g) * O + (o0 + o)) * c.L + l) * c.n) + quad;
      *dst = v;
    }
  }
}

// Multi-group MAC: for each limb and coefficient k the accumulators form a small
// matrix product Acc_k[g][o] = sum_i Pt_k[g][i] * C_k[i][o].  One CTA takes 32
// consecutive coefficients of one limb, GC groups and all O outputs; P is walked in
// chunks of IC plaintexts staged in shared memory with cp.async (double buffered),
// so the model is read from HBM once per group block.  Warp (wg, wo) owns groups
// wg*GT.. and outputs wo*OT..; its lanes are the 32 coefficients, so every shared
// load is one conflict-free 128-byte row.
__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, bool ok) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
               "r"(ok ? 16 : 0));
}

// A chunked pass (several calls over plaintext ranges) reads plaintexts
// [mi0, mi0 + cnt) of the model against a plaintext buffer of pP plaintexts per group
// and adds into the accumulators (accum != 0) instead of overwriting them.
template <int GT, int OT, bool CMP>
__global__ void __launch_bounds__(512) k_mac_tiled(DevCtx c, const uint32_t* __restrict__ pt,
                                                   const uint32_t* __restrict__ model,
                                                   uint32_t* __restrict__ acc, int G, int GC,
                                                   int IC, int pP, int mi0, int cnt, int accum) {
  extern __shared__ __align__(16) uint32_t sm[];
  const uint32_t l = blockIdx.y, k0 = blockIdx.x * 32;
  const int g0 = blockIdx.z * GC;
  const int O = 2 * (int)c.Kp;
  const int WO = (O + OT - 1) / OT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wg = warp / WO, wo = warp - wg * WO;
  const int rows = GC + O;                 // rows of 32 words per plaintext index
  const int buf_words = IC * rows * 32;
  const uint32_t p = c.mq[l].p;
  const uint64_t mu = c.mq[l].mu;
  const size_t n = c.n, L = c.L, P = (size_t)pP;
  const uint32_t CNT = (uint32_t)cnt;

  // copy slots: slot q = rr * 8 + piece (row rr of a staged plaintext index, 16-byte
  // piece, shared-memory word offset 4 q) belongs to thread q mod blockDim for every
  // plaintext of a chunk, so its source address is formed once per chunk and advanced
  // by a fixed stride; rows * 8 <= 4 * blockDim is checked by the launcher
  // the compact model stores c0 only ([P][O/2][L][n]); its c1 rows are generated
  const size_t pt_stride = L * n;
  const size_t model_stride = (size_t)(CMP ? O / 2 : O) * L * n;
  auto load_chunk = [&](int b, uint32_t i0) {
    uint32_t* dst = sm + b * buf_words;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int q = threadIdx.x + k * blockDim.x;
      if (q < rows * 8) {
        const int rr = q >> 3, piece = q & 7;
        const bool is_pt = rr < GC;
        const int o = rr - GC;
        if (!is_pt && CMP && (o & 1)) continue;  // c1: generated below
        const bool gok = !is_pt || g0 + rr < G;
        const size_t stride = is_pt ? pt_stride : model_stride;
        const int mrow = CMP ? o >> 1 : o;
        const uint32_t* src =
            is_pt ? pt + ((size_t)(gok ? g0 + rr : 0) * P * L + l) * n + k0 + piece * 4
                  : model + ((size_t)mrow * L + l) * n + k0 + piece * 4 +
                        (size_t)mi0 * model_stride;
        src += (size_t)i0 * stride;
        for (int ii = 0; ii < IC; ii++, src += stride) {
          const bool ok = gok && i0 + ii < CNT;
          cp_async16_zfill(dst + ii * rows * 32 + 4 * q, ok ? src : pt, ok);
        }
      }
    }
    if (CMP) {
      // c1 of model ciphertext (i, j') at device position k of limb l: 64-bit word
      // l n + k of the stream (model seed, domain 8, i Kp + j') mod q_l; one ChaCha20
      // block gives the 8 coefficients of an item (plaintext, j', 8 of the 32 columns)
      const int kp = O / 2, items = IC * kp * 4;
      for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int ii = it / (kp * 4), rem = it - ii * kp * 4, jp = rem >> 2, cb = rem & 3;
        uint32_t* d = dst + ii * rows * 32 + (GC + 2 * jp + 1) * 32 + 8 * cb;
        const uint32_t li = i0 + ii;
        if (li < CNT) {
          uint32_t w[16];
          chacha_block(c.model_seed, 8, (uint64_t)(mi0 + li) * kp + jp,
                       (uint32_t)(((size_t)l * n + k0 + 8 * cb) / 8), w);
#pragma unroll
          for (int u = 0; u < 8; u++)
            d[u] = red64((uint64_t)w[2 * u] | ((uint64_t)w[2 * u + 1] << 32), p, mu);
        } else {
#pragma unroll
          for (int u = 0; u < 8; u++) d[u] = 0;
        }
      }
    }
    asm volatile("cp.async.commit_group;\n");
  };

  // 64-bit accumulators: each product (< 2^60) is added as one 64-bit multiply-add
  // (no carry flag shared between accumulators, so their chains interleave), and the
  // sums are reduced once per staged chunk (IC <= 15 products on top of a reduced value
  // stay below 2^64)
  uint64_t a64[GT][OT];
#pragma unroll
  for (int x = 0; x < GT; x++)
#pragma unroll
    for (int y = 0; y < OT; y++) a64[x][y] = 0;
  const int gb = wg * GT, ob = wo * OT;
  const int nchunks = (int)((CNT + IC - 1) / IC);
  load_chunk(0, 0);
  for (int ch = 0; ch < nchunks; ch++) {
    if (ch + 1 < nchunks) {
      load_chunk((ch + 1) & 1, (ch + 1) * IC);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    const uint32_t* buf = sm + (ch & 1) * buf_words;
    const int iend = min(IC, (int)CNT - ch * IC);
#pragma unroll 3
    for (int ii = 0; ii < iend; ii++) {
      const uint32_t* rowp = buf + ii * rows * 32 + lane;
      uint32_t x[GT], y[OT];
#pragma unroll
      for (int g = 0; g < GT; g++) x[g] = rowp[(gb + g < GC ? gb + g : 0) * 32];
#pragma unroll
      for (int o = 0; o < OT; o++) y[o] = rowp[(GC + (ob + o < O ? ob + o : 0)) * 32];
#pragma unroll
      for (int g = 0; g < GT; g++)
#pragma unroll
        for (int o = 0; o < OT; o++) a64[g][o] += (uint64_t)x[g] * y[o];
    }
#pragma unroll
    for (int g = 0; g < GT; g++)
#pragma unroll
      for (int o = 0; o < OT; o++) a64[g][o] = red64(a64[g][o], p, mu);
    __syncthreads();  // the buffer is refilled two chunks later
  }
#pragma unroll
  for (int g = 0; g < GT; g++) {
    const int gg = g0 + gb + g;
    if (gb + g >= GC || gg >= G) continue;
#pragma unroll
    for (int o = 0; o < OT; o++) {
      if (ob + o >= O) continue;
      uint32_t* a = acc + (((size_t)gg * O + ob + o) * L + l) * n + k0 + lane;
      *a = accum ? csub(*a + (uint32_t)a64[g][o], p) : (uint32_t)a64[g][o];
    }
  }
}

// acc[x] = sum_split partial[split][x] mod q_l, x over G*O*L*n words
__global__ void k_mac_reduce(DevCtx c, const uint32_t* __restrict__ partial, int splits,
                             size_t words, uint32_t* __restrict__ acc) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= words) return;
  const uint32_t l = (uint32_t)((x >> c.logn) % c.L);
  uint64_t s = 0;
  for (int k = 0; k < splits; k++) s += __ldg(partial + (size_t)k * words + x);
  acc[x] = red64(s, c.mq[l].p, c.mq[l].mu);
}

// ------------------------------------------------------------------ rotations
// resident CTAs of at most 256 threads the key-switch kernels are compiled for: three
// (80 registers) at n = 8192, two (128 registers) at n = 16384, where the transform
// passes need more; smaller rings launch fewer threads and need no bound
constexpr int ks_min_blocks(int logn) { return logn == 13 ? 3 : logn >= 14 ? 2 : 1; }
// pass schedule of the key-switch and export transforms: radix-32 passes last (the
// schedule the encoder's autotuner picks at n = 8192 and 16384)
constexpr int KS_PLAN = 2;

// digits[ct][i][:] = tau_g(INTT_{q_i}(c1 limb i)): the RNS digits of the rotated c1 as
// integer polynomials with coefficients in [0, q_i).  The automorphism X -> X^g is
// applied in the coefficient domain at the output (coefficient k moves to k g mod 2n,
// negated when that is n or more), so the input is read contiguously; the result
// equals INTT_{q_i} of the NTT-domain permutation of c1.
template <int LOGN>
__global__ void __launch_bounds__(256, ks_min_blocks(LOGN))
    k_ks_digits(DevCtx c, const uint32_t* __restrict__ acc, uint32_t* __restrict__ digits,
                uint32_t gal) {
  constexpr uint32_t N = 1u << LOGN;
  extern __shared__ uint32_t sm[];
  const uint32_t ct = blockIdx.x, i = blockIdx.y;
  const uint32_t* src = acc + ((size_t)(ct * 2 + 1) * c.L + i) * N;
  uint32_t* dst = digits + ((size_t)ct * c.L + i) * N;
  const uint32_t q = c.mq[i].p;
  // coalesced 16-byte loads into the padded buffer (the first inverse pass reads 32
  // consecutive words per thread, which straight from global memory would be strided)
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  for (uint32_t k = threadIdx.x; k < N / 4; k += blockDim.x) {
    const uint4 v = __ldg(&s4[k]);
    uint32_t* w = sm + padi(4 * k);  // the 4 words never straddle a pad word
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  }
  __syncthreads();
  const auto st = [=](uint32_t k, uint32_t v) {
    const uint32_t e = (k * gal) & (2 * N - 1);
    if (e < N) dst[e] = v;
    else dst[e - N] = v ? q - v : 0;
  };
  ntt_inv_io<LOGN, SmemLd, decltype(st), KS_PLAN>(sm, c.mq[i], SmemLd{sm}, st);
}

// Key switch and add, one thread-block cluster of L - 1 CTAs per (ciphertext, target
// limb l).  Cluster rank i owns RNS digit d = i (i < l) or i + 1 (i >= l) and holds
// X_d = NTT_l(d-th digit) in its shared memory; the digit l needs no transform, its
// NTT_l is tau(acc1 limb l) itself.  Rank i then produces its 1/(L - 1) slice of the
// coefficients, reading every rank's X_d through distributed shared memory and
// tau(acc1 limb l) from global memory, each multiplied by its key parts:
//   out[ct][0][l] = acc0 + tau(acc0) + sum_d X_d * k0[d][l],
//   out[ct][1][l] = acc1 + sum_d X_d * k1[d][l].
// One transform buffer per CTA (the products are formed in the reduction).
// gkj: [L digits][L limbs][4][n] = (k0, k0 Shoup, k1, k1 Shoup), NTT domain.
template <int LOGN>
__global__ void __launch_bounds__(256, ks_min_blocks(LOGN))
    k_ks_cluster(DevCtx c, const uint32_t* __restrict__ acc,
                 const uint32_t* __restrict__ digits, const uint32_t* __restrict__ gkj,
                 uint32_t* __restrict__ out, uint32_t gal) {
  constexpr uint32_t N = 1u << LOGN;
  extern __shared__ uint32_t sm[];
  uint32_t* x = sm;  // padded transform buffer
  cg::cluster_group cluster = cg::this_cluster();
  const uint32_t i = blockIdx.x, l = blockIdx.y, ct = blockIdx.z;
  const uint32_t L = c.L, R = L - 1;  // cluster ranks
  const ModP m = c.mq[l];
  const uint32_t p = m.p;
  const uint32_t* c1 = acc + ((size_t)(ct * 2 + 1) * c.L + l) * N;
  {
    const uint32_t d = i < l ? i : i + 1;
    const uint32_t* dg = digits + ((size_t)ct * c.L + d) * N;
    const auto ld = [=](uint32_t kk) { return csub(__ldg(&dg[kk]), p); };  // d < 2 q_l
    ntt_fwd_io<LOGN, decltype(ld), SmemSt, KS_PLAN>(x, m, ld, SmemSt{x});
  }
  cluster.sync();
  const uint32_t slice = (N + R - 1) / R;
  const uint32_t j0 = i * slice, j1 = min(N, j0 + slice);
  const uint32_t* c0 = acc + ((size_t)(ct * 2 + 0) * c.L + l) * N;
  uint32_t* o0 = out + ((size_t)(ct * 2 + 0) * c.L + l) * N;
  uint32_t* o1 = out + ((size_t)(ct * 2 + 1) * c.L + l) * N;
  const uint32_t* kl = gkj + ((size_t)l * L + l) * 4 * N;  // key parts of digit l
  // every rank's transform buffer and key parts, resolved once
  const uint32_t* xr[EPHDC_MAXL - 1];
  const uint32_t* kr[EPHDC_MAXL - 1];
#pragma unroll
  for (uint32_t r = 0; r < EPHDC_MAXL - 1; r++) {
    xr[r] = r < R ? cluster.map_shared_rank(x, r) : x;
    kr[r] = gkj + ((size_t)(r < l ? r : r + 1) * L + l) * 4 * N;
  }
  // the products accumulate in 64 bits: every factor is below q_l < 2^30, so the L
  // products (< 2^60 each) and the two added words stay below 2^63 and are reduced
  // once; only the key parts k0, k1 are read (not their Shoup quotients)
  for (uint32_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const uint32_t gp = galois_pos(j, gal, LOGN);
    uint64_t s0 = (uint64_t)__ldg(&c0[j]) + __ldg(&c0[gp]);
    uint64_t s1 = __ldg(&c1[j]);
    // every rank's loads issued before the first product (L is at most EPHDC_MAXL)
    const uint32_t vl = __ldg(&c1[gp]);
    const uint32_t k0l = __ldg(kl + j), k1l = __ldg(kl + 2 * N + j);
    uint32_t v[EPHDC_MAXL - 1], k0[EPHDC_MAXL - 1], k1[EPHDC_MAXL - 1];
    const uint32_t pj = padi(j);
#pragma unroll
    for (uint32_t r = 0; r < EPHDC_MAXL - 1; r++) {
      if (r < R) {
        v[r] = xr[r][pj];
        k0[r] = __ldg(kr[r] + j);
        k1[r] = __ldg(kr[r] + 2 * N + j);
      }
    }
    s0 += (uint64_t)vl * k0l;
    s1 += (uint64_t)vl * k1l;
#pragma unroll
    for (uint32_t r = 0; r < EPHDC_MAXL - 1; r++) {
      if (r < R) {
        s0 += (uint64_t)v[r] * k0[r];
        s1 += (uint64_t)v[r] * k1[r];
      }
    }
    o0[j] = red64(s0, p, m.mu);
    o1[j] = red64(s1, p, m.mu);
  }
  cluster.sync();  // keep every CTA's shared memory alive until all slices are read
}

// ------------------------------------------------------------------ export
// out[ct][poly][l] = INTT_l(acc[ct][poly][l])
template <int LOGN>
__global__ void __launch_bounds__(512) k_export(DevCtx c, const uint32_t* __restrict__ acc,
                                                uint32_t* __restrict__ out) {
  constexpr uint32_t N = 1u << LOGN;
  extern __shared__ uint32_t sm[];
  const uint32_t item = blockIdx.x;  // (ct*2 + poly)*L + l
  const uint32_t l = item % c.L;
  const uint32_t* src = acc + (size_t)item * N;
  uint32_t* dst = out + (size_t)item * N;
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  for (uint32_t k = threadIdx.x; k < N / 4; k += blockDim.x) {
    const uint4 v = __ldg(&s4[k]);
    uint32_t* w = sm + padi(4 * k);  // the 4 words never straddle a pad word
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  }
  __syncthreads();
  const auto st = [=](uint32_t k, uint32_t v) { dst[k] = v; };
  ntt_inv_io<LOGN, SmemLd, decltype(st), KS_PLAN>(sm, c.mq[l], SmemLd{sm}, st);
}

inline unsigned ntt_threads(const DevCtx& c) {
  unsigned t = c.n / 32;
  return t < 64 ? 64 : (t > 512 ? 512 : t);
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

namespace ephdc {

cudaError_t launch_encode_plain(const DevCtx& c, const int8_t* H, int B, uint32_t* pt,
                                cudaStream_t st, uint32_t i0, uint32_t ni) {
  const int G = (B + c.cap - 1) / c.cap;
  if (ni == 0) {
    i0 = 0;
    ni = c.P;
  }
  if (ni != c.P && (c.layout || c.scale_g)) return cudaErrorNotSupported;
  const size_t smem = encode_smem_bytes(c.logn);
  // at most 256 threads: at n = 16384 two CTAs per SM (compact coefficient copy)
  const unsigned threads = ntt_threads(c) < 256 ? ntt_threads(c) : 256;
  EPHDC_DISPATCH_LOGN(c.logn, LG, {
    auto kern = c.ntt_plan == 1 ? k_encode_plain<LG, 1>
              : c.ntt_plan == 2 ? k_encode_plain<LG, 2> : k_encode_plain<LG, 0>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<G * ni, threads, smem, st>>>(c, H, B, pt, i0, ni);
  });
  if (c.scale_g) k_scale_plain<<<G * c.P, 256, 0, st>>>(c, pt);
  return cudaGetLastError();
}

// the tiled kernel's instantiations: (groups per warp, outputs per warp)
template <int GT, int OT>
static cudaError_t run_mac_tiled(const DevCtx& c, const uint32_t* pt, int G, const uint32_t* model,
                                 uint32_t* acc, int GC, int IC, int pP, int mi0, int cnt,
                                 int accum, cudaStream_t st) {
  // IC <= 15 keeps (reduced value) + IC products below 2^64 between reductions
  const int O = 2 * c.Kp;
  // no wider group block than the groups present
  const int Gr = (G + GT - 1) / GT * GT;
  if (GC > Gr) GC = Gr;
  if (IC > 15) IC = 15;
  const int warps = (GC / GT) * ((O + OT - 1) / OT);
  const size_t smem = 2 * (size_t)IC * (GC + O) * 32 * sizeof(uint32_t);
  if (warps < 1 || warps > 16 || GC % GT || (GC + O) * 8 > 4 * warps * 32)
    return cudaErrorInvalidConfiguration;
  auto kern = c.compact ? k_mac_tiled<GT, OT, true> : k_mac_tiled<GT, OT, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(c.n / 32, c.L, (G + GC - 1) / GC);
  kern<<<grid, warps * 32, smem, st>>>(c, pt, model, acc, G, GC, IC, pP, mi0, cnt, accum);
  return cudaGetLastError();
}

cudaError_t launch_mac_tiled(const DevCtx& c, const uint32_t* pt, int G, const uint32_t* model,
                             uint32_t* acc, const MacTiling& t, cudaStream_t st, int pP, int mi0,
                             int cnt, int accum) {
  if (pP <= 0) pP = cnt = (int)c.P;  // the whole pass
  switch (t.gt * 100 + t.ot) {
#define EPHDC_TILED(GT_, OT_)                                                              \
  case GT_ * 100 + OT_:                                                                    \
    return run_mac_tiled<GT_, OT_>(c, pt, G, model, acc, t.gc, t.ic, pP, mi0, cnt, accum, st);
    EPHDC_TILED(2, 4)
    EPHDC_TILED(2, 7)
    EPHDC_TILED(2, 8)
    EPHDC_TILED(4, 4)
    EPHDC_TILED(4, 7)
    EPHDC_TILED(4, 8)
#undef EPHDC_TILED
    default: return cudaErrorInvalidConfiguration;
  }
}

cudaError_t launch_mac(const DevCtx& c, const uint32_t* pt, int G, const uint32_t* model,
                       uint32_t* partial, int splits_max, uint32_t* acc, cudaStream_t st) {
  constexpr int OC = 4;
  const int O = 2 * c.Kp;
  // same rule as the scratch sizing: enough (limb, quad, split) threads to fill
  // every SM a few times over
  long per_split = (long)c.L * (c.n / 4) * G;
  long s = (152L * 2048 + per_split - 1) / per_split;
  if (s > (long)c.P) s = c.P;
  if (s > 64) s = 64;
  if (s > splits_max) s = splits_max;
  if (s < 1) s = 1;
  const int splits = (int)s;
  const unsigned threads = 256;
  const unsigned blocks = (c.L * (c.n / 4) + threads - 1) / threads;
  for (int o0 = 0; o0 < O; o0 += OC) {
    const int nout = O - o0 < OC ? O - o0 : OC;
    k_mac<OC><<<dim3(blocks, G, splits), threads, 0, st>>>(c, pt, model, partial, G, splits, o0,
                                                           nout);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_mac_reduce(c, partial, splits, (size_t)G * O * c.L * c.n, acc, st);
}

cudaError_t launch_mac_reduce(const DevCtx& c, const uint32_t* partial, int splits, size_t words,
                              uint32_t* acc, cudaStream_t st) {
  k_mac_reduce<<<(unsigned)((words + 255) / 256), 256, 0, st>>>(c, partial, splits, words, acc);
  return cudaGetLastError();
}

cudaError_t launch_rotate_sum(const DevCtx& c, uint32_t* acc, uint32_t* tmp, uint32_t* digits,
                              int count, const uint32_t* gk, cudaStream_t st) {
  const size_t smem1 = padded_words(c.n) * sizeof(uint32_t);
  const size_t smem2 = padded_words(c.n) * sizeof(uint32_t);
  // at most 256 threads per CTA (see ks_min_blocks)
  const unsigned ks_threads = ntt_threads(c) < 256 ? ntt_threads(c) : 256;
  uint32_t* cur = acc;
  uint32_t* nxt = tmp;
  const size_t gk_step = (size_t)c.L * c.L * 4 * c.n;
  uint32_t gal[32];
  for (uint32_t j = 0; j < c.logr; j++) {  // 3^(W 2^j) mod 2n
    uint64_t r = 1, b = 3, ex = (uint64_t)c.W << j, mod = 2ull * c.n;
    while (ex) {
      if (ex & 1) r = r * b % mod;
      b = b * b % mod;
      ex >>= 1;
    }
    gal[j] = (uint32_t)r;
  }
  EPHDC_DISPATCH_LOGN(c.logn, LG, {
    cudaError_t e = set_smem(k_ks_digits<LG>, smem1);
    if (e == cudaSuccess) e = set_smem(k_ks_cluster<LG>, smem2);
    if (e != cudaSuccess) return e;
    for (uint32_t j = 0; j < c.logr; j++) {
      k_ks_digits<LG><<<dim3(count, c.L), ks_threads, smem1, st>>>(c, cur, digits, gal[j]);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(c.L - 1, c.L, count);
      cfg.blockDim = dim3(ks_threads);
      cfg.dynamicSmemBytes = smem2;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = c.L - 1;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, k_ks_cluster<LG>, c, (const uint32_t*)cur,
                             (const uint32_t*)digits, gk + j * gk_step, nxt, gal[j]);
      if (e != cudaSuccess) return e;
      uint32_t* t = cur;
      cur = nxt;
      nxt = t;
    }
  });
  return cudaGetLastError();
}

cudaError_t launch_export(const DevCtx& c, const uint32_t* acc, int count, uint32_t* out,
                          cudaStream_t st) {
  const size_t smem = padded_words(c.n) * sizeof(uint32_t);
  EPHDC_DISPATCH_LOGN(c.logn, LG, {
    cudaError_t e = set_smem(k_export<LG>, smem);
    if (e != cudaSuccess) return e;
    k_export<LG><<<count * 2 * c.L, ntt_threads(c), smem, st>>>(c, acc, out);
  });
  return cudaGetLastError();
}

}  // namespace ephdc
