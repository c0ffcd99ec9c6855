// Server-side and checking kernels: key generation, secret-key encryption of the
// class hypervectors (Sec. 4.1: the model is encrypted once and shipped), score
// decryption, and conversions of device NTT-domain objects to the coefficient
// domain.  Randomness is the ChaCha20 stream of RFC 8439 keyed by the seed:
//   domain 1: secret s (word k mod 3 -> {0, 1, -1})
//   domain 2/3: uniform a / Gaussian e of model ciphertext number i*Kp + jp
//   domain 4/5: uniform a / Gaussian e of Galois key (fold step j, digit i), obj j<<16|i
// A uniform coefficient (limb l, index k) is 64-bit word l*n + k mod q_l; a Gaussian
// coefficient k inverts the cumulative table at 64-bit word k.
#include <cuda_fp16.h>

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

__device__ __forceinline__ uint32_t galois_pos(uint32_t j, uint32_t g, uint32_t logn) {
  const uint32_t n2mask = (2u << logn) - 1;
  const uint32_t e = 2 * brev(j, logn) + 1;
  return brev((((e * g) & n2mask) - 1) >> 1, logn);
}

// ------------------------------------------------------------------ keygen
// sk[l] = NTT_l(s mod q_l)
__global__ void __launch_bounds__(512) k_secret(DevCtx c, uint64_t seed, uint32_t* __restrict__ sk) {
  extern __shared__ uint32_t sm[];
  const uint32_t l = blockIdx.x, p = c.mq[l].p;
  for (uint32_t b = threadIdx.x; b < c.n / 16; b += blockDim.x) {
    uint32_t w[16];
    chacha_block(seed, 1, 0, b, w);
#pragma unroll
    for (int u = 0; u < 16; u++) {
      const uint32_t v = w[u] % 3u;
      sm[padi(b * 16 + u)] = v == 2 ? p - 1 : v;
    }
  }
  __syncthreads();
  ntt_fwd_smem(sm, c.logn, c.mq[l]);
  for (uint32_t j = threadIdx.x; j < c.n; j += blockDim.x) sk[(size_t)l * c.n + j] = sm[padi(j)];
}

// gk[j][i][l] = (k0, Shoup(k0), k1, Shoup(k1)):  k1 = a,  k0 = -a s + e + [i == l] tau_gj(s)
__global__ void __launch_bounds__(512) k_galois_keys(DevCtx c, uint64_t seed,
                                                     const uint32_t* __restrict__ sk,
                                                     uint32_t* __restrict__ gk) {
  extern __shared__ uint32_t sm[];
  uint32_t* ab = sm;
  uint32_t* eb = sm + padded_words(c.n);
  const uint32_t j = blockIdx.x / c.L, i = blockIdx.x % c.L, l = blockIdx.y;
  const ModP m = c.mq[l];
  const uint64_t obj = ((uint64_t)j << 16) | i;
  fill_uniform(c, seed, 4, obj, l, ab);
  fill_gauss(c, seed, 5, obj, m.p, eb);
  __syncthreads();
  ntt_fwd_smem(ab, c.logn, m);
  ntt_fwd_smem(eb, c.logn, m);
  const uint32_t gal = c.galois[j];
  const uint32_t* s = sk + (size_t)l * c.n;
  uint32_t* dst = gk + (((size_t)j * c.L + i) * c.L + l) * 4 * c.n;
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) {
    const uint32_t a = ab[padi(x)];
    uint32_t k0 = subm(eb[padi(x)], mulm(a, s[x], m), m.p);
    if (i == l) k0 = addm(k0, s[galois_pos(x, gal, c.logn)], m.p);
    dst[x] = k0;
    dst[c.n + x] = (uint32_t)(((uint64_t)k0 << 32) / m.p);
    dst[2 * c.n + x] = a;
    dst[3 * c.n + x] = (uint32_t)(((uint64_t)a << 32) / m.p);
  }
}

// digit v of residue `val` (balanced base 256: byte v of val + 0x80808080, less 128) as
// the fp16 element of the digit model, for v < 4
__device__ __forceinline__ void store_digits(const DevCtx& c, uint16_t* mdig, uint32_t i,
                                             uint32_t o, uint32_t l, uint32_t x, uint32_t val) {
  const uint32_t vb = val + 0x80808080u;
#pragma unroll
  for (uint32_t v = 0; v < 4; v++)
    mdig[mdig_index(c.n, c.P, mdig_rows(c.Kp), i, o, v, l, x)] =
        __half_as_ushort(__int2half_rn((int)((vb >> (8 * v)) & 255u) - 128));
}

// ------------------------------------------------------------------ model encryption
// One CTA per (ciphertext i*Kp + jp, limb l).  Class value c_{jp*k_in+jin}[i*r+ch] fills
// slot (rho, ch*W + jin*cap_row + qq) for all qq < cap_row; encode with the inverse NTT
// mod t; c1 = a, c0 = -a s + e + round(q m / t).
__global__ void __launch_bounds__(512) k_encrypt_model(DevCtx c, const int8_t* __restrict__ cls,
                                                       const uint32_t* __restrict__ sk,
                                                       uint64_t seed, uint32_t* __restrict__ model) {
  extern __shared__ uint32_t sm[];
  uint32_t* mb = sm;
  uint32_t* ab = sm + padded_words(c.n);
  uint32_t* eb = ab + padded_words(c.n);
  const uint32_t cidx = blockIdx.x, l = blockIdx.y;
  const uint32_t i = cidx / c.Kp, jp = cidx - i * c.Kp;
  const uint32_t half = c.n >> 1;
  const ModP m = c.mq[l];
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
  // c1: the standard model draws a in the coefficient domain (domain 2) and transforms
  // it; the compact model draws it in the evaluation domain at device position k
  // (domain 8, word l n + k), so that the multiply-accumulate can regenerate it
  if (c.compact) fill_uniform(c, c.model_seed, 8, cidx, l, ab);
  else fill_uniform(c, seed, 2, cidx, l, ab);
  fill_gauss(c, seed, 3, cidx, m.p, eb);
  __syncthreads();
  ntt_inv_smem(mb, c.logn, c.mt);  // m in [0, t)
  // the scaled message round(q m / t) is formed per coefficient (it is not linear in
  // m), then transformed with a and e
  const ScaledMsg scaled(c, l);
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) mb[padi(x)] = scaled(mb[padi(x)]);
  __syncthreads();
  ntt_fwd_smem(mb, c.logn, m);
  if (!c.compact) ntt_fwd_smem(ab, c.logn, m);
  ntt_fwd_smem(eb, c.logn, m);
  const uint32_t* s = sk + (size_t)l * c.n;
  uint32_t* c0 = model + ((size_t)(cidx * 2 + 0) * c.L + l) * c.n;
  uint32_t* c1 = model + ((size_t)(cidx * 2 + 1) * c.L + l) * c.n;
  const uint32_t O = 2 * c.Kp;
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) {
    const uint32_t a = ab[padi(x)];
    uint32_t v = subm(eb[padi(x)], mulm(a, s[x], m), m.p);
    v = addm(v, mb[padi(x)], m.p);
    if (c.compact) {  // c0 only, [P][O/2][L][n]
      model[((size_t)cidx * c.L + l) * c.n + x] = v;
    } else if (c.mdig) {  // the signed base-256 digits of c0 and c1 as fp16 operand rows
      store_digits(c, reinterpret_cast<uint16_t*>(model), i, jp * 2, l, x, v);
      store_digits(c, reinterpret_cast<uint16_t*>(model), i, jp * 2 + 1, l, x, a);
    } else if (c.layout) {  // outputs o = j' * 2 + poly of plaintext i
      model[blk_index(c.n, c.P, O, i, jp * 2, l, x)] = v;
      model[blk_index(c.n, c.P, O, i, jp * 2 + 1, l, x)] = a;
    } else {
      c0[x] = v;
      c1[x] = a;
    }
  }
}

// ------------------------------------------------------------------ seeded model message
// One CTA per (model ciphertext, limb): c0 from the coefficient-domain message into the
// NTT domain, and c1 = a regenerated from the ChaCha20 stream the encryption drew it
// from (domain 2, ciphertext number), then transformed.
__global__ void __launch_bounds__(512) k_model_from_seeded(DevCtx c,
                                                           const uint32_t* __restrict__ c0w,
                                                           uint64_t seed,
                                                           uint32_t* __restrict__ model) {
  extern __shared__ uint32_t sm[];
  uint32_t* b0 = sm;
  uint32_t* b1 = sm + padded_words(c.n);
  const uint32_t cidx = blockIdx.x, l = blockIdx.y;
  const ModP m = c.mq[l];
  const uint32_t* src = c0w + ((size_t)cidx * c.L + l) * c.n;
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) b0[padi(x)] = src[x];
  fill_uniform(c, seed, 2, cidx, l, b1);
  __syncthreads();
  ntt_fwd_smem(b0, c.logn, m);
  ntt_fwd_smem(b1, c.logn, m);
  uint32_t* c0 = model + ((size_t)(cidx * 2 + 0) * c.L + l) * c.n;
  uint32_t* c1 = model + ((size_t)(cidx * 2 + 1) * c.L + l) * c.n;
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) {
    c0[x] = b0[padi(x)];
    c1[x] = b1[padi(x)];
  }
}

// ------------------------------------------------------------------ decryption (check)
// xbuf[ct][l] = INTT_l(c0 + c1 * s)
__global__ void __launch_bounds__(512) k_dec_phase(DevCtx c, const uint32_t* __restrict__ ct,
                                                   const uint32_t* __restrict__ sk,
                                                   uint32_t* __restrict__ xbuf) {
  extern __shared__ uint32_t sm[];
  const uint32_t item = blockIdx.x, l = blockIdx.y;
  const ModP m = c.mq[l];
  const uint32_t* c0 = ct + ((size_t)(item * 2 + 0) * c.L + l) * c.n;
  const uint32_t* c1 = ct + ((size_t)(item * 2 + 1) * c.L + l) * c.n;
  // the score ciphertexts are in the coefficient domain: transform both to NTT
  uint32_t* b0 = sm;
  uint32_t* b1 = sm + padded_words(c.n);
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) {
    b0[padi(x)] = c0[x];
    b1[padi(x)] = c1[x];
  }
  __syncthreads();
  ntt_fwd_smem(b1, c.logn, m);
  const uint32_t* s = sk + (size_t)l * c.n;
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) b1[padi(x)] = mulm(b1[padi(x)], s[x], m);
  __syncthreads();
  ntt_inv_smem(b1, c.logn, m);
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x)
    xbuf[((size_t)item * c.L + l) * c.n + x] = addm(b0[padi(x)], b1[padi(x)], m.p);
}

__device__ void big_add(uint32_t* a, const uint32_t* b) {
  uint64_t cr = 0;
  for (int i = 0; i < EPHDC_BIGW; i++) {
    uint64_t v = (uint64_t)a[i] + b[i] + cr;
    a[i] = (uint32_t)v;
    cr = v >> 32;
  }
}
__device__ bool big_ge(const uint32_t* a, const uint32_t* b) {
  for (int i = EPHDC_BIGW - 1; i >= 0; i--)
    if (a[i] != b[i]) return a[i] > b[i];
  return true;
}
__device__ void big_sub(uint32_t* a, const uint32_t* b) {
  int64_t br = 0;
  for (int i = 0; i < EPHDC_BIGW; i++) {
    int64_t v = (int64_t)a[i] - b[i] - br;
    br = v < 0;
    a[i] = (uint32_t)(v + (br ? (1ll << 32) : 0));
  }
}

// one thread per coefficient of each score ciphertext: CRT of the phase limbs, then
// round(t x / Q) mod t, written over limb 0 of the coefficient (only this thread reads
// that coefficient's limbs)
__global__ void __launch_bounds__(256) k_dec_round(DevCtx c, uint32_t* __restrict__ xbuf) {
  const uint32_t item = blockIdx.x;
  const uint32_t x = blockIdx.y * blockDim.x + threadIdx.x;
  if (x >= c.n) return;
  uint32_t X[EPHDC_BIGW] = {0};
  for (uint32_t l = 0; l < c.L; l++) {
    const uint32_t y = mulm(xbuf[((size_t)item * c.L + l) * c.n + x], c.qhat_inv[l], c.mq[l]);
    uint32_t term[EPHDC_BIGW];
    uint64_t cr = 0;
    for (int w = 0; w < EPHDC_BIGW; w++) {
      uint64_t v = (uint64_t)c.big_Qhat[l][w] * y + cr;
      term[w] = (uint32_t)v;
      cr = v >> 32;
    }
    big_add(X, term);
  }
  while (big_ge(X, c.big_Q)) big_sub(X, c.big_Q);
  // num = t X + floor(Q/2); quotient bit by bit (it is at most t)
  uint64_t cr = 0;
  for (int w = 0; w < EPHDC_BIGW; w++) {
    uint64_t v = (uint64_t)X[w] * c.t + cr;
    X[w] = (uint32_t)v;
    cr = v >> 32;
  }
  big_add(X, c.big_Qhalf);
  uint32_t quo = 0;
  for (int b = 31 - __clz(c.t); b >= 0; b--) {
    uint32_t Qs[EPHDC_BIGW];
    for (int w = 0; w < EPHDC_BIGW; w++) {
      uint64_t v = ((uint64_t)c.big_Q[w] << b);
      uint32_t lo = (uint32_t)v;
      uint32_t carry_in = (w > 0 && b > 0) ? (c.big_Q[w - 1] >> (32 - b)) : 0;
      Qs[w] = lo | carry_in;
    }
    if (big_ge(X, Qs)) {
      big_sub(X, Qs);
      quo |= 1u << b;
    }
  }
  xbuf[(size_t)item * c.L * c.n + x] = quo % c.t;
}

// one CTA per score ciphertext: the rounded coefficients back to slots with the
// forward NTT mod t, then the score slots
__global__ void __launch_bounds__(512) k_dec_scores(DevCtx c, const uint32_t* __restrict__ xbuf,
                                                    int B, uint32_t* __restrict__ scores) {
  extern __shared__ uint32_t sm[];
  const uint32_t item = blockIdx.x;
  const uint32_t g = item / c.Kp, jp = item - g * c.Kp;
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x)
    sm[padi(x)] = xbuf[(size_t)item * c.L * c.n + x];
  __syncthreads();
  ntt_fwd_smem(sm, c.logn, c.mt);  // coefficients -> slots (device order)
  const uint32_t half = c.n >> 1;
  const uint32_t per = 2 * c.cap_row * c.k_in;
  for (uint32_t u = threadIdx.x; u < per; u += blockDim.x) {
    const uint32_t rho = u / (c.cap_row * c.k_in);
    const uint32_t rest = u - rho * c.cap_row * c.k_in;
    const uint32_t jin = rest / c.cap_row, qq = rest - jin * c.cap_row;
    const uint64_t beta = (uint64_t)g * c.cap + rho * c.cap_row + qq;
    if (beta >= (uint64_t)B) continue;
    const uint32_t sidx = rho * half + jin * c.cap_row + qq;
    scores[beta * c.k + jp * c.k_in + jin] = sm[padi(__ldg(&c.slot2pos[sidx]))];
  }
}

// ------------------------------------------------------------------ conversions
// out[(item*nsub + sub)*L + l] = INTT_l(in + item*istride + sub*sstride + l*lstride)
__global__ void __launch_bounds__(512) k_to_coeff(DevCtx c, const uint32_t* __restrict__ in,
                                                  uint32_t* __restrict__ out, int nsub, int istride,
                                                  int sstride, int lstride) {
  extern __shared__ uint32_t sm[];
  const uint32_t item = blockIdx.x, sub = blockIdx.y, l = blockIdx.z;
  const uint32_t* src = in + (size_t)item * istride + (size_t)sub * sstride + (size_t)l * lstride;
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) sm[padi(x)] = src[x];
  __syncthreads();
  ntt_inv_smem(sm, c.logn, c.mq[l]);
  uint32_t* dst = out + (((size_t)item * nsub + sub) * c.L + l) * c.n;
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) dst[x] = sm[padi(x)];
}

__global__ void __launch_bounds__(512) k_sk_coeff(DevCtx c, const uint32_t* __restrict__ sk,
                                                  int32_t* __restrict__ out) {
  extern __shared__ uint32_t sm[];
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) sm[padi(x)] = sk[x];
  __syncthreads();
  ntt_inv_smem(sm, c.logn, c.mq[0]);
  const uint32_t p = c.mq[0].p;
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) {
    const uint32_t v = sm[padi(x)];
    out[x] = v > p / 2 ? (int32_t)v - (int32_t)p : (int32_t)v;
  }
}

// natural-order transform: a_hat[j] = a(psi^(2j+1)) sits at device position brv(j)
__global__ void __launch_bounds__(512) k_ntt_natural(DevCtx c, uint32_t limb, uint32_t* poly,
                                                     int inverse) {
  extern __shared__ uint32_t sm[];
  const ModP m = limb < c.L ? c.mq[limb] : c.mt;
  uint32_t* a = poly + (size_t)blockIdx.x * c.n;
  if (!inverse) {
    for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) sm[padi(x)] = a[x];
    __syncthreads();
    ntt_fwd_smem(sm, c.logn, m);
    for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) a[x] = sm[padi(brev(x, c.logn))];
  } else {
    for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) sm[padi(brev(x, c.logn))] = a[x];
    __syncthreads();
    ntt_inv_smem(sm, c.logn, m);
    for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) a[x] = sm[padi(x)];
  }
}

// compact model [P][O/2][L][n] (c0 only) -> the whole model [P][O/2][2][L][n] with c1
// regenerated from the model seed (host-format conversions)
__global__ void k_expand_compact(DevCtx c, const uint32_t* __restrict__ c0,
                                 uint32_t* __restrict__ full, size_t blocks) {
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < blocks;
       x += (size_t)gridDim.x * blockDim.x) {
    const uint32_t b = (uint32_t)(x % (c.n / 8));
    size_t rest = x / (c.n / 8);
    const uint32_t l = (uint32_t)(rest % c.L);
    const size_t cidx = rest / c.L;
    uint32_t w[16];
    chacha_block(c.model_seed, 8, cidx, (uint32_t)(((size_t)l * c.n) / 8 + b), w);
    const uint32_t* src = c0 + (cidx * c.L + l) * c.n + 8 * b;
    uint32_t* d0 = full + ((cidx * 2) * c.L + l) * c.n + 8 * b;
    uint32_t* d1 = full + ((cidx * 2 + 1) * c.L + l) * c.n + 8 * b;
#pragma unroll
    for (int u = 0; u < 8; u++) {
      d0[u] = src[u];
      d1[u] = red64((uint64_t)w[2 * u] | ((uint64_t)w[2 * u + 1] << 32), c.mq[l].p,
                    c.mq[l].mu);
    }
  }
}

// standard [P][O][L][n] -> digit model (the padding is zeroed by the launcher)
__global__ void k_todigits(DevCtx c, const uint32_t* __restrict__ src, uint16_t* __restrict__ mdig,
                           size_t words) {
  const uint32_t O = 2 * c.Kp;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < words;
       x += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(x % c.n);
    size_t rest = x / c.n;
    const uint32_t l = (uint32_t)(rest % c.L);
    rest /= c.L;
    const uint32_t o = (uint32_t)(rest % O), i = (uint32_t)(rest / O);
    store_digits(c, mdig, i, o, l, k, src[x]);
  }
}

// digit model -> standard [P][O][L][n]: residue = sum_v d_v 2^(8v) (exact: the digits
// of a residue in [0, q_l) reassemble it)
__global__ void k_undigit(DevCtx c, const uint16_t* __restrict__ mdig, uint32_t* __restrict__ dst,
                          size_t words) {
  const uint32_t O = 2 * c.Kp;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < words;
       x += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(x % c.n);
    size_t rest = x / c.n;
    const uint32_t l = (uint32_t)(rest % c.L);
    rest /= c.L;
    const uint32_t o = (uint32_t)(rest % O), i = (uint32_t)(rest / O);
    int64_t r = 0;
    for (uint32_t v = 0; v < 4; v++)
      r += (int64_t)__half2int_rn(
               __ushort_as_half(mdig[mdig_index(c.n, c.P, mdig_rows(c.Kp), i, o, v, l, k)]))
           << (8 * v);
    dst[x] = (uint32_t)r;
  }
}

// blocked [L][n/4][A][B][4] -> standard [A][B][L][n] (host-format conversions)
__global__ void k_unblock(DevCtx c, const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                          uint32_t A, uint32_t B, size_t words) {
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < words;
       x += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(x % c.n);
    size_t rest = x / c.n;
    const uint32_t l = (uint32_t)(rest % c.L);
    rest /= c.L;
    const uint32_t b = (uint32_t)(rest % B), a = (uint32_t)(rest / B);
    dst[x] = src[blk_index(c.n, A, B, a, b, l, k)];
  }
}

}  // namespace

namespace ephdc {

cudaError_t launch_keygen(const DevCtx& c, uint64_t seed, uint32_t* sk, uint32_t* gk,
                          cudaStream_t st) {
  const size_t s1 = padded_words(c.n) * 4, s2 = 2 * padded_words(c.n) * 4;
  cudaError_t e = set_smem(k_secret, s1);
  if (e == cudaSuccess) e = set_smem(k_galois_keys, s2);
  if (e != cudaSuccess) return e;
  k_secret<<<c.L, ntt_threads(c), s1, st>>>(c, seed, sk);
  if (c.logr) k_galois_keys<<<dim3(c.logr * c.L, c.L), ntt_threads(c), s2, st>>>(c, seed, sk, gk);
  return cudaGetLastError();
}

cudaError_t launch_encrypt_model(const DevCtx& c, const int8_t* classes, const uint32_t* sk,
                                 uint64_t seed, uint32_t* model, cudaStream_t st) {
  const size_t s = 3 * padded_words(c.n) * 4;
  cudaError_t e = set_smem(k_encrypt_model, s);
  if (e != cudaSuccess) return e;
  if (c.mdig) {  // the digit model's padding rows and plaintexts are zero
    e = cudaMemsetAsync(model, 0, mdig_bytes(c.n, c.L, c.P, c.Kp), st);
    if (e != cudaSuccess) return e;
  }
  k_encrypt_model<<<dim3(c.P * c.Kp, c.L), ntt_threads(c), s, st>>>(c, classes, sk, seed, model);
  return cudaGetLastError();
}

cudaError_t launch_decrypt_scores(const DevCtx& c, const uint32_t* sk, const uint32_t* ct, int B,
                                  uint32_t* xbuf, uint32_t* scores, cudaStream_t st) {
  const int count = ((B + c.cap - 1) / c.cap) * c.Kp;
  const size_t s2 = 2 * padded_words(c.n) * 4, s1 = padded_words(c.n) * 4;
  cudaError_t e = set_smem(k_dec_phase, s2);
  if (e == cudaSuccess) e = set_smem(k_dec_scores, s1);
  if (e != cudaSuccess) return e;
  k_dec_phase<<<dim3(count, c.L), ntt_threads(c), s2, st>>>(c, ct, sk, xbuf);
  k_dec_round<<<dim3(count, (c.n + 255) / 256), 256, 0, st>>>(c, xbuf);
  k_dec_scores<<<count, ntt_threads(c), s1, st>>>(c, xbuf, B, scores);
  return cudaGetLastError();
}

cudaError_t launch_model_to_seeded(const DevCtx& c, const uint32_t* model, uint32_t* c0w,
                                  cudaStream_t st) {
  // c0 of every model ciphertext ([P*Kp][2][L][n], NTT domain) to [P*Kp][L][n] coefficients
  return launch_to_coeff(c, model, c0w, (int)(c.P * c.Kp), 1, (int)(2 * c.L * c.n), (int)c.n, 0,
                         st);
}

cudaError_t launch_model_from_seeded(const DevCtx& c, const uint32_t* c0w, uint64_t seed,
                                    uint32_t* model, cudaStream_t st) {
  const size_t smem = 2 * padded_words(c.n) * 4;
  cudaError_t e = set_smem(k_model_from_seeded, smem);
  if (e != cudaSuccess) return e;
  k_model_from_seeded<<<dim3(c.P * c.Kp, c.L), ntt_threads(c), smem, st>>>(c, c0w, seed, model);
  return cudaGetLastError();
}

cudaError_t launch_decrypt_phases(const DevCtx& c, uint32_t* xbuf, int count, int B,
                                  uint32_t* scores, cudaStream_t st) {
  const size_t s1 = padded_words(c.n) * 4;
  cudaError_t e = set_smem(k_dec_scores, s1);
  if (e != cudaSuccess) return e;
  k_dec_round<<<dim3(count, (c.n + 255) / 256), 256, 0, st>>>(c, xbuf);
  k_dec_scores<<<count, ntt_threads(c), s1, st>>>(c, xbuf, B, scores);
  return cudaGetLastError();
}

cudaError_t launch_expand_compact(const DevCtx& c, const uint32_t* c0, uint32_t* full,
                                  cudaStream_t st) {
  const size_t blocks = (size_t)c.P * c.Kp * c.L * (c.n / 8);
  const unsigned grid = (unsigned)((blocks + 255) / 256 < 152 * 32 ? (blocks + 255) / 256 : 152 * 32);
  k_expand_compact<<<grid, 256, 0, st>>>(c, c0, full, blocks);
  return cudaGetLastError();
}

cudaError_t launch_model_to_digits(const DevCtx& c, const uint32_t* model, uint16_t* mdig,
                                   cudaStream_t st) {
  const size_t words = (size_t)c.P * 2 * c.Kp * c.L * c.n;
  cudaError_t e =
      cudaMemsetAsync(mdig, 0, mdig_bytes(c.n, c.L, c.P, c.Kp), st);
  if (e != cudaSuccess) return e;
  k_todigits<<<1024, 256, 0, st>>>(c, model, mdig, words);
  return cudaGetLastError();
}

cudaError_t launch_undigit(const DevCtx& c, const uint16_t* mdig, uint32_t* model,
                           cudaStream_t st) {
  const size_t words = (size_t)c.P * 2 * c.Kp * c.L * c.n;
  k_undigit<<<1024, 256, 0, st>>>(c, mdig, model, words);
  return cudaGetLastError();
}

cudaError_t launch_unblock(const DevCtx& c, const uint32_t* src, uint32_t* dst, uint32_t A,
                           uint32_t B, cudaStream_t st) {
  const size_t words = (size_t)A * B * c.L * c.n;
  const unsigned blocks = (unsigned)((words + 255) / 256 < 152 * 32 ? (words + 255) / 256 : 152 * 32);
  k_unblock<<<blocks, 256, 0, st>>>(c, src, dst, A, B, words);
  return cudaGetLastError();
}

cudaError_t launch_to_coeff(const DevCtx& c, const uint32_t* in, uint32_t* out, int count,
                            int nsub, int istride, int lstride, int digit_major,
                            cudaStream_t st) {
  // digit_major: Galois-key layout [j][i][l][4][n] with k0 at slot 0 and k1 at slot 2
  const size_t s = padded_words(c.n) * 4;
  cudaError_t e = set_smem(k_to_coeff, s);
  if (e != cudaSuccess) return e;
  const int sstride = digit_major ? 2 * (int)c.n : (int)c.L * (int)c.n;
  k_to_coeff<<<dim3(count, nsub, c.L), ntt_threads(c), s, st>>>(c, in, out, nsub, istride,
                                                                 sstride, lstride);
  return cudaGetLastError();
}

cudaError_t launch_sk_to_coeff(const DevCtx& c, const uint32_t* sk, int32_t* out, uint32_t*,
                               cudaStream_t st) {
  const size_t s = padded_words(c.n) * 4;
  cudaError_t e = set_smem(k_sk_coeff, s);
  if (e != cudaSuccess) return e;
  k_sk_coeff<<<1, ntt_threads(c), s, st>>>(c, sk, out);
  return cudaGetLastError();
}

cudaError_t launch_ntt_natural(const DevCtx& c, uint32_t limb, uint32_t* poly, int count,
                               int inverse, cudaStream_t st) {
  const size_t s = padded_words(c.n) * 4;
  cudaError_t e = set_smem(k_ntt_natural, s);
  if (e != cudaSuccess) return e;
  k_ntt_natural<<<count, ntt_threads(c), s, st>>>(c, limb, poly, inverse);
  return cudaGetLastError();
}

}  // namespace ephdc
