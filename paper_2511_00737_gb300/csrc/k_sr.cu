// Server-side variant of HDC inference (HE-HDC-SR, Sec. 3): the client encrypts its
// query hypervectors in the SIMD form and sends them; the server multiplies them by
// the class hypervectors held as plaintexts and sums over the dimensions, then the
// rotations and the export are those of the client-side path.  This is the method
// the client-runtime comparison of Sec. 6 (Table t:clientrt) sets EP-HDC against.
//
// Randomness (ChaCha20, RFC 8439, keyed by the seed): query ciphertext number
// gi = g*P + i draws its uniform a from domain 6 and its Gaussian e from domain 7,
// with the same word-to-coefficient rules as the model encryption.
#include "ephdc_internal.cuh"

namespace {

inline unsigned ntt_threads(const DevCtx& c) {
  unsigned t = c.n / 32;
  return t < 64 ? 64 : (t > 512 ? 512 : t);
}
template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ------------------------------------------------------------------ query encryption
// One CTA per query ciphertext (g, i): the slots of query plaintext (g, i) are packed
// as in the client-side encoder, the inverse NTT mod t gives m in [0, t), and per limb
//   c0 = NTT(round(Q m / t) + e) - NTT(a) * s,   c1 = NTT(a)
// (the NTT is linear, so NTT(round(Q m / t) + e) is one transform).  e (|e| <= 19) is drawn
// once and kept as bytes; both transforms of a limb finish in shared memory and the
// ciphertext is written with 16-byte stores.
template <int LOGN, int V>
__global__ void __launch_bounds__(LOGN >= 14 ? 512 : 256, LOGN >= 14 ? 1 : 2)
    k_encrypt_queries(DevCtx c, const int8_t* __restrict__ H, int B,
                      const uint32_t* __restrict__ sk, uint64_t seed,
                      uint32_t* __restrict__ ctq) {
  constexpr uint32_t N = 1u << LOGN;
  extern __shared__ uint32_t sm[];
  uint32_t* mb = sm;
  uint32_t* wb = mb + padded_words(N);
  uint32_t* vb = wb + padded_words(N);
  int8_t* eb = reinterpret_cast<int8_t*>(vb + padded_words(N));
  const uint32_t gi = blockIdx.x;
  const uint32_t g = gi / c.P, i = gi - g * c.P;
  for (uint32_t j = threadIdx.x; j < N; j += blockDim.x) mb[padi(j)] = 0;
  for (uint32_t b = threadIdx.x; b < N / 8; b += blockDim.x) {
    uint32_t w[16];
    chacha_block(seed, 7, gi, b, w);
#pragma unroll
    for (int u = 0; u < 8; u++)
      eb[b * 8 + u] = (int8_t)cdt_sample(c, (uint64_t)w[2 * u] | ((uint64_t)w[2 * u + 1] << 32));
  }
  __syncthreads();
  pack_query_slots(c, H, B, g, i, mb);
  __syncthreads();
  ntt_inv_t<LOGN, V, false>(mb, c.mt);  // slots (scaled by n^-1) -> m in [0, t)
  for (uint32_t l = 0; l < c.L; l++) {
    const ModP m = c.mq[l];
    const uint32_t p = m.p;
    const ScaledMsg sm_l(c, l);
    auto dm_e = [=](uint32_t k) -> uint32_t {
      const int32_t e = eb[k];
      return addm(sm_l(mb[padi(k)]), e < 0 ? (uint32_t)((int32_t)p + e) : (uint32_t)e, p);
    };
    ntt_fwd_io<LOGN, decltype(dm_e), SmemSt, V>(wb, m, dm_e, SmemSt{vb});
    fill_uniform(c, seed, 6, gi, l, wb);
    __syncthreads();
    ntt_fwd_t<LOGN, V>(wb, m);
    const uint4* s4 = reinterpret_cast<const uint4*>(sk + (size_t)l * N);
    uint4* c0 = reinterpret_cast<uint4*>(ctq + (((size_t)gi * 2 + 0) * c.L + l) * N);
    uint4* c1 = reinterpret_cast<uint4*>(ctq + (((size_t)gi * 2 + 1) * c.L + l) * N);
    for (uint32_t k = threadIdx.x; k < N / 4; k += blockDim.x) {
      const uint4 s = __ldg(s4 + k);
      const uint4 a = make_uint4(wb[padi(4 * k)], wb[padi(4 * k + 1)], wb[padi(4 * k + 2)],
                                 wb[padi(4 * k + 3)]);
      uint4 v;
      v.x = subm(vb[padi(4 * k)], mulm(a.x, s.x, m), p);
      v.y = subm(vb[padi(4 * k + 1)], mulm(a.y, s.y, m), p);
      v.z = subm(vb[padi(4 * k + 2)], mulm(a.z, s.z, m), p);
      v.w = subm(vb[padi(4 * k + 3)], mulm(a.w, s.w, m), p);
      c0[k] = v;
      c1[k] = a;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ plaintext model
// One CTA per model plaintext (jp, i): class value c_{jp*k_in+jin}[i*r+ch] fills slot
// (rho, ch*W + jin*cap_row + qq) for all qq < cap_row (the model side of the SIMD
// layout), the inverse NTT mod t encodes it, and each limb stores NTT(lift(m)).
// mm: [Kp][P][L][n], the layout of a client-side plaintext batch with Kp groups.
__global__ void __launch_bounds__(512) k_encode_model_plain(DevCtx c,
                                                            const int8_t* __restrict__ cls,
                                                            uint32_t* __restrict__ mm) {
  extern __shared__ uint32_t sm[];
  uint32_t* mb = sm;
  uint32_t* wb = sm + padded_words(c.n);
  const uint32_t cidx = blockIdx.x;
  const uint32_t jp = cidx / c.P, i = cidx - jp * c.P;
  const uint32_t half = c.n >> 1;
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) {
    const uint32_t sidx = __ldg(&c.pos2slot[x]);
    const uint32_t rho = sidx >= half;
    const uint32_t col = sidx - rho * half;
    const uint32_t ch = col / c.W, within = col - ch * c.W;
    const uint32_t jin = within / c.cap_row;
    uint32_t v = 0;
    const uint32_t d = i * c.r + ch;
    if (jin < c.k_in && d < c.D) {
      const int h = cls[(size_t)(jp * c.k_in + jin) * c.D + d];
      v = h < 0 ? (uint32_t)(h + (int)c.t) : (uint32_t)h;
    }
    mb[padi(x)] = v;
  }
  __syncthreads();
  ntt_inv_smem(mb, c.logn, c.mt);
  const uint32_t t = c.t, thalf = (t - 1) / 2;
  for (uint32_t l = 0; l < c.L; l++) {
    const ModP m = c.mq[l];
    const uint32_t p = m.p;
    for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) {
      const uint32_t v = mb[padi(x)];
      wb[padi(x)] = v <= thalf ? v : v + p - t;
    }
    __syncthreads();
    ntt_fwd_smem(wb, c.logn, m);
    // the scaling operation folded into plaintext i (as on the client-side path)
    const uint32_t w = c.scale_g ? scale_factor(c, l, c.P / c.scale_g - i / c.scale_g) : 1;
    uint32_t* dst = mm + ((size_t)cidx * c.L + l) * c.n;
    for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x)
      dst[x] = w == 1 ? wb[padi(x)] : mulm(wb[padi(x)], w, m);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ ct x pt MAC
// partial[split][g][jp*2+poly][l][n] = sum_{i in split} ctq[g][i][poly][l] * mm[jp][i][l]
// (mod q_l).  A thread owns 4 consecutive coefficients of one limb of one group, both
// polynomials and OC classes; it reads each query-ciphertext word once and each
// model-plaintext word once per group.  Products (< 2^60) accumulate in 64 bits and
// are reduced every 15 terms.
template <int OC>
__global__ void __launch_bounds__(256) k_ctpt_mac(DevCtx c, const uint32_t* __restrict__ ctq,
                                                  const uint32_t* __restrict__ mm,
                                                  uint32_t* __restrict__ partial, int G,
                                                  int splits, int j0, int nj) {
  const uint32_t quads = c.n >> 2;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= c.L * quads) return;
  const uint32_t l = tid / quads, quad = tid - l * quads;
  const uint32_t g = blockIdx.y, split = blockIdx.z;
  const uint32_t per = (c.P + splits - 1) / splits;
  const uint32_t i0 = split * per, i1 = min(c.P, i0 + per);
  const uint32_t p = c.mq[l].p;
  const uint64_t mu = c.mq[l].mu;
  const size_t limb_q = (size_t)c.L * quads;  // uint4 per (object, poly)
  uint64_t acc[2][OC][4];
#pragma unroll
  for (int po = 0; po < 2; po++)
#pragma unroll
    for (int o = 0; o < OC; o++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[po][o][e] = 0;
  // ctq[g][i][poly][l]: uint4 index ((g*P + i)*2 + poly) * L*quads + l*quads + quad
  const uint4* cp = reinterpret_cast<const uint4*>(ctq) + (size_t)g * c.P * 2 * limb_q +
                    (size_t)l * quads + quad;
  // mm[jp][i][l]: uint4 index (jp*P + i) * L*quads + l*quads + quad
  const uint4* mp = reinterpret_cast<const uint4*>(mm) + (size_t)l * quads + quad;
  const size_t jp_step = (size_t)c.P * limb_q;
  uint32_t cnt = 0;
  for (uint32_t i = i0; i < i1; i++) {
    const uint4 a0 = __ldg(cp + (size_t)i * 2 * limb_q);
    const uint4 a1 = __ldg(cp + ((size_t)i * 2 + 1) * limb_q);
#pragma unroll
    for (int o = 0; o < OC; o++) {
      if (o < nj) {
        const uint4 b = __ldg(mp + (size_t)(j0 + o) * jp_step + (size_t)i * limb_q);
        acc[0][o][0] += (uint64_t)a0.x * b.x;
        acc[0][o][1] += (uint64_t)a0.y * b.y;
        acc[0][o][2] += (uint64_t)a0.z * b.z;
        acc[0][o][3] += (uint64_t)a0.w * b.w;
        acc[1][o][0] += (uint64_t)a1.x * b.x;
        acc[1][o][1] += (uint64_t)a1.y * b.y;
        acc[1][o][2] += (uint64_t)a1.z * b.z;
        acc[1][o][3] += (uint64_t)a1.w * b.w;
      }
    }
    if (++cnt == 15) {
      cnt = 0;
#pragma unroll
      for (int po = 0; po < 2; po++)
#pragma unroll
        for (int o = 0; o < OC; o++)
#pragma unroll
          for (int e = 0; e < 4; e++) acc[po][o][e] = red64(acc[po][o][e], p, mu);
    }
  }
  const uint32_t O = 2 * c.Kp;
#pragma unroll
  for (int o = 0; o < OC; o++) {
    if (o < nj) {
#pragma unroll
      for (int po = 0; po < 2; po++) {
        const uint4 v = make_uint4(red64(acc[po][o][0], p, mu), red64(acc[po][o][1], p, mu),
                                   red64(acc[po][o][2], p, mu), red64(acc[po][o][3], p, mu));
        const uint32_t out = (j0 + o) * 2 + po;
        uint4* dst = reinterpret_cast<uint4*>(
            partial + ((((size_t)split * G + g) * O + out) * c.L + l) * c.n) + quad;
        *dst = v;
      }
    }
  }
}

}  // namespace

namespace ephdc {

cudaError_t launch_encrypt_queries(const DevCtx& c, const int8_t* H, int B, const uint32_t* sk,
                                   uint64_t seed, uint32_t* ctq, cudaStream_t st) {
  const int G = (B + c.cap - 1) / c.cap;
  const size_t smem = 3 * padded_words(c.n) * sizeof(uint32_t) + c.n;
  EPHDC_DISPATCH_LOGN(c.logn, LG, {
    auto kern = c.ntt_plan == 1 ? k_encrypt_queries<LG, 1>
              : c.ntt_plan == 2 ? k_encrypt_queries<LG, 2> : k_encrypt_queries<LG, 0>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<G * c.P, ntt_threads(c), smem, st>>>(c, H, B, sk, seed, ctq);
  });
  return cudaGetLastError();
}

cudaError_t launch_encode_model_plain(const DevCtx& c, const int8_t* classes, uint32_t* mm,
                                      cudaStream_t st) {
  const size_t smem = 2 * padded_words(c.n) * sizeof(uint32_t);
  cudaError_t e = set_smem(k_encode_model_plain, smem);
  if (e != cudaSuccess) return e;
  k_encode_model_plain<<<c.Kp * c.P, ntt_threads(c), smem, st>>>(c, classes, mm);
  return cudaGetLastError();
}

cudaError_t launch_ctpt_mac(const DevCtx& c, const uint32_t* ctq, int G, const uint32_t* mm,
                            uint32_t* partial, int splits_max, uint32_t* acc, cudaStream_t st) {
  constexpr int OC = 4;
  // enough (limb, quad, split) threads to fill every SM a few times over
  long per_split = (long)c.L * (c.n / 4) * G;
  long s = (152L * 2048 + per_split - 1) / per_split;
  if (s > (long)c.P) s = c.P;
  if (s > 64) s = 64;
  if (s > splits_max) s = splits_max;
  if (s < 1) s = 1;
  const int splits = (int)s;
  const unsigned threads = 256;
  const unsigned blocks = (c.L * (c.n / 4) + threads - 1) / threads;
  for (int j0 = 0; j0 < (int)c.Kp; j0 += OC) {
    const int nj = (int)c.Kp - j0 < OC ? (int)c.Kp - j0 : OC;
    k_ctpt_mac<OC><<<dim3(blocks, G, splits), threads, 0, st>>>(c, ctq, mm, partial, G, splits,
                                                               j0, nj);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_mac_reduce(c, partial, splits, (size_t)G * 2 * c.Kp * c.L * c.n, acc, st);
}

}  // namespace ephdc
