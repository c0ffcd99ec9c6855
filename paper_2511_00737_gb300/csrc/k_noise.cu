// The noise-growth experiment of Sec. 5.2 (Alg. 1, findDmax): how many plaintext x
// ciphertext products can be accumulated before decryption goes wrong, for a given
// ring degree and plaintext modulus.  One trial evaluates the client-side dot product
// for every prefix length D' = 1..D at once: the accumulator after D' products is
// the prefix sum of the products, so its decryption is the evaluation with D'
// dimensions.  D_i of the trial is the number of leading prefixes that decrypt to
// the clear dot products mod t.
//
// Steps (one group of queries, one class, the paper's layout k_in = k = 1, r = 1):
//   1. phase of every prefix in the NTT domain, X_D' = sum_{i < D'} pt_i (c0_i + c1_i s),
//      as a chunked scan over i (local prefix sums, chunk totals, offsets);
//   2. inverse NTT of every prefix phase, in place;
//   3. CRT, rounding and decoding of every prefix (the checking decryption kernel);
//   4. the first prefix whose score differs from the clear prefix sum for any query.
#include "ephdc_internal.cuh"

namespace {

inline unsigned ntt_threads(const DevCtx& c) {
  unsigned t = c.n / 32;
  return t < 64 ? 64 : (t > 512 ? 512 : t);
}

// local prefix sums over chunk blockIdx.y of [0, D): X[i][l][x] for i in the chunk,
// and the chunk's total in T[chunk][l][x]
__global__ void __launch_bounds__(256) k_prefix_local(DevCtx c, const uint32_t* __restrict__ pt,
                                                      const uint32_t* __restrict__ model,
                                                      const uint32_t* __restrict__ sk, int D,
                                                      int chunk, uint32_t* __restrict__ X,
                                                      uint32_t* __restrict__ T) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= c.L * c.n) return;
  const uint32_t l = tid / c.n, x = tid - l * c.n;
  const ModP m = c.mq[l];
  const uint32_t s = sk[(size_t)l * c.n + x];
  const int i0 = blockIdx.y * chunk, i1 = min(D, i0 + chunk);
  const size_t ln = (size_t)c.L * c.n;
  uint32_t acc = 0;
  for (int i = i0; i < i1; i++) {
    const uint32_t c0 = model[((size_t)i * 2 + 0) * ln + tid];
    const uint32_t c1 = model[((size_t)i * 2 + 1) * ln + tid];
    const uint32_t ph = addm(c0, mulm(c1, s, m), m.p);
    acc = addm(acc, mulm(pt[(size_t)i * ln + tid], ph, m), m.p);
    X[(size_t)i * ln + tid] = acc;
  }
  T[(size_t)blockIdx.y * ln + tid] = acc;
}

// adds the totals of all earlier chunks to every prefix of chunk blockIdx.y + 1
__global__ void __launch_bounds__(256) k_prefix_offset(DevCtx c, int D, int chunk,
                                                       const uint32_t* __restrict__ T,
                                                       uint32_t* __restrict__ X) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= c.L * c.n) return;
  const uint32_t l = tid / c.n;
  const uint32_t p = c.mq[l].p;
  const size_t ln = (size_t)c.L * c.n;
  const int ch = blockIdx.y + 1;
  uint32_t off = 0;
  for (int e = 0; e < ch; e++) off = addm(off, T[(size_t)e * ln + tid], p);
  const int i0 = ch * chunk, i1 = min(D, i0 + chunk);
  for (int i = i0; i < i1; i++) X[(size_t)i * ln + tid] = addm(X[(size_t)i * ln + tid], off, p);
}

// in-place inverse NTT of X[i][l]
__global__ void __launch_bounds__(512) k_prefix_coeff(DevCtx c, uint32_t* X) {
  extern __shared__ uint32_t sm[];
  const uint32_t i = blockIdx.x, l = blockIdx.y;
  uint32_t* poly = X + ((size_t)i * c.L + l) * c.n;
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) sm[padi(x)] = poly[x];
  __syncthreads();
  ntt_inv_smem(sm, c.logn, c.mq[l]);
  for (uint32_t x = threadIdx.x; x < c.n; x += blockDim.x) poly[x] = sm[padi(x)];
}

// first[0] = min over queries of the first prefix index whose decrypted score differs
// from sum_{i <= d} h[q][i] c[i] mod t (scores[d][q], one class)
__global__ void __launch_bounds__(256) k_first_wrong(DevCtx c, const int8_t* __restrict__ H,
                                                     const int8_t* __restrict__ cls, int B, int D,
                                                     const uint32_t* __restrict__ scores,
                                                     int* __restrict__ first) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B) return;
  const int64_t t = c.t;
  int64_t clear = 0;
  for (int d = 0; d < D; d++) {
    if ((d & 255) == 0 && d >= *(volatile int*)first) return;
    clear = (clear + (int64_t)H[(size_t)q * D + d] * cls[d]) % t;
    const uint32_t want = (uint32_t)(clear < 0 ? clear + t : clear);
    if (scores[(size_t)d * c.cap + q] != want) {
      atomicMin(first, d);
      return;
    }
  }
}

}  // namespace

namespace ephdc {

int prefix_chunks(const DevCtx& c, int D) {
  // about 152 x 2048 threads in flight: chunks of the scan over i
  int chunks = (int)((152L * 2048 + (long)c.L * c.n - 1) / ((long)c.L * c.n));
  if (chunks > D) chunks = D;
  if (chunks < 1) chunks = 1;
  const int chunk = (D + chunks - 1) / chunks;
  return (D + chunk - 1) / chunk;
}

// T: prefix_chunks(c, D) x L x n words of scratch
cudaError_t launch_prefix_phases(const DevCtx& c, const uint32_t* pt, const uint32_t* model,
                                 const uint32_t* sk, int D, uint32_t* X, uint32_t* T,
                                 cudaStream_t st) {
  const unsigned threads = 256;
  const unsigned blocks = (c.L * c.n + threads - 1) / threads;
  int chunks = prefix_chunks(c, D);
  const int chunk = (D + chunks - 1) / chunks;
  k_prefix_local<<<dim3(blocks, chunks), threads, 0, st>>>(c, pt, model, sk, D, chunk, X, T);
  if (chunks > 1)
    k_prefix_offset<<<dim3(blocks, chunks - 1), threads, 0, st>>>(c, D, chunk, T, X);
  const size_t smem = padded_words(c.n) * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(k_prefix_coeff, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_prefix_coeff<<<dim3(D, c.L), ntt_threads(c), smem, st>>>(c, X);
  return cudaGetLastError();
}

cudaError_t launch_first_wrong(const DevCtx& c, const int8_t* H, const int8_t* cls, int B, int D,
                               const uint32_t* scores, int* first, cudaStream_t st) {
  k_first_wrong<<<(B + 255) / 256, 256, 0, st>>>(c, H, cls, B, D, scores, first);
  return cudaGetLastError();
}

}  // namespace ephdc
