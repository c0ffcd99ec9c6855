// HDC encoding (Sec. 2.1 random projection) with the quantiser of Sec. 5.1 fused
// into the epilogue:  H = clamp(floor((X Wt^T + 2^(s-1)) / 2^s), -2^(b-1), 2^(b-1)-1).
//
// X [B][F] and Wt [D][F] are int8 with F contiguous, so both operands are K-major.
// The product runs on the INT8 tensor-core path that sm_103a accepts (mma.sync
// m16n8k32 s8 x s8 -> s32; the tcgen05 kind::i8 form is not available on this
// target), which is exact: |A| <= 128 * F < 2^31.  Tiles are staged with cp.async
// through a 3-stage shared-memory ring with 16-byte padded rows (conflict-free
// 32-bit fragment loads).
#include "ephdc_internal.cuh"

namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 3, ROWB = BK + 16;
constexpr int SMEM_BYTES = STAGES * (BM + BN) * ROWB;

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
               "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void mma_s8(int* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(256) k_hdc(DevCtx c, const int8_t* __restrict__ X,
                                             const int8_t* __restrict__ Wt, int B,
                                             int8_t* __restrict__ H) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * BM * ROWB;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int F = (int)c.F, D = (int)c.D;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps, 64 x 32 each
  const int nk = (F + BK - 1) / BK;

  auto load_stage = [&](int stage, int kt) {
#pragma unroll
    for (int it = 0; it < 2; it++) {
      const int idx = threadIdx.x + it * 256;
      const int row = idx >> 2, ch = idx & 3;
      const int kb = kt * BK + ch * 16;
      const int gr = m0 + row, gc = n0 + row;
      const bool oka = gr < B && kb < F, okb = gc < D && kb < F;
      cp_async16(sA + (stage * BM + row) * ROWB + ch * 16, oka ? X + (size_t)gr * F + kb : X,
                 oka ? 16 : 0);
      cp_async16(sB + (stage * BN + row) * ROWB + ch * 16, okb ? Wt + (size_t)gc * F + kb : Wt,
                 okb ? 16 : 0);
    }
  };

  int acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[a][b][e] = 0;

#pragma unroll
  for (int s = 0; s < STAGES - 1; s++) {
    if (s < nk) load_stage(s, s);
    cp_async_commit();
  }
  for (int kt = 0; kt < nk; kt++) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    const int nxt = kt + STAGES - 1;
    if (nxt < nk) load_stage(nxt % STAGES, nxt);
    cp_async_commit();
    const uint8_t* a = sA + (kt % STAGES) * BM * ROWB;
    const uint8_t* b = sB + (kt % STAGES) * BN * ROWB;
#pragma unroll
    for (int ks = 0; ks < BK / 32; ks++) {
      const int kb = ks * 32 + (lane & 3) * 4;
      uint32_t af[4][4], bf[4][2];
#pragma unroll
      for (int mt = 0; mt < 4; mt++) {
        const int r = wm * 64 + mt * 16 + (lane >> 2);
        af[mt][0] = *reinterpret_cast<const uint32_t*>(a + r * ROWB + kb);
        af[mt][1] = *reinterpret_cast<const uint32_t*>(a + (r + 8) * ROWB + kb);
        af[mt][2] = *reinterpret_cast<const uint32_t*>(a + r * ROWB + kb + 16);
        af[mt][3] = *reinterpret_cast<const uint32_t*>(a + (r + 8) * ROWB + kb + 16);
      }
#pragma unroll
      for (int nt = 0; nt < 4; nt++) {
        const int cc = wn * 32 + nt * 8 + (lane >> 2);
        bf[nt][0] = *reinterpret_cast<const uint32_t*>(b + cc * ROWB + kb);
        bf[nt][1] = *reinterpret_cast<const uint32_t*>(b + cc * ROWB + kb + 16);
      }
#pragma unroll
      for (int mt = 0; mt < 4; mt++)
#pragma unroll
        for (int nt = 0; nt < 4; nt++) mma_s8(acc[mt][nt], af[mt], bf[nt]);
    }
  }
  cp_async_wait<0>();

  const int s = c.shift;
  const int rnd = s > 0 ? 1 << (s - 1) : 0;
  const int lo = -(1 << (c.bits - 1)), hi = (1 << (c.bits - 1)) - 1;
#pragma unroll
  for (int mt = 0; mt < 4; mt++)
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int row = m0 + wm * 64 + mt * 16 + (lane >> 2) + h * 8;
        const int col = n0 + wn * 32 + nt * 8 + (lane & 3) * 2;
        if (row >= B) continue;
#pragma unroll
        for (int e = 0; e < 2; e++) {
          if (col + e >= D) continue;
          int v = (acc[mt][nt][h * 2 + e] + rnd) >> s;  // arithmetic shift = floor
          v = v < lo ? lo : (v > hi ? hi : v);
          H[(size_t)row * D + col + e] = (int8_t)v;
        }
      }
}

}  // namespace

namespace ephdc {

cudaError_t launch_hdc_encode(const DevCtx& c, const int8_t* X, const int8_t* Wt, int B,
                              int8_t* H, cudaStream_t st) {
  cudaError_t e =
      cudaFuncSetAttribute(k_hdc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  dim3 grid((c.D + BN - 1) / BN, (B + BM - 1) / BM);
  k_hdc<<<grid, 256, SMEM_BYTES, st>>>(c, X, Wt, B, H);
  return cudaGetLastError();
}

}  // namespace ephdc
