// Dense multiply-accumulate of many groups on the tensor cores (the batch x classes
// contraction of Sec. 4.1's HE compute when many query groups share the model):
//   Acc_k[g][o] = sum_i Pt_k[g][i] * C_k[i][o]  (mod q_l)   for every coefficient k.
//
// Exact byte split: residues < 2^30 are written as 4 bytes, a = sum_u a_u 2^(8u),
// c = sum_v c_v 2^(8v), so sum_i a c = sum_{u,v} 2^(8(u+v)) S_uv with
// S_uv = sum_i a_u c_v.  Per coefficient one MMA computes every S_uv at once:
// rows (u, g) of the digit matrix A' (4 GP x K) times columns (v, o) of B' (K x 4 OP).
// Bytes are fp16 values, products are < 2^16, and a window of 256 plaintexts keeps
// every fp32 partial sum below 2^24: exact.  After each window the TMEM accumulator
// is read out: the 4 digit rows (u, g) of a group sit in one warp (lanes u*8 + g mod
// 8), so each thread weights its S_uv by 2^(8(u+v)) mod q_l and sums over v in
// registers, two shuffles sum over u, and the owner lane adds the result into the
// group's accumulators (reduced mod q_l every window; no atomics).  The next window
// restarts the MMA.
//
// One CTA: limb l, KB consecutive coefficients, one block of GP groups, all outputs.
// Per 16-plaintext chunk: cp.async stages the raw residues (rows of KB words) into a
// 4-deep ring; 8 warps split them into fp16 digits laid out as the MMA's canonical
// K-major, no-swizzle operand tiles (double buffered); one thread issues
// tcgen05.mma (M = 128, N = 4 OP, K = 16) per coefficient and M tile, and commits to
// the buffer's mbarrier.  All waits are bounded.
#include <cuda_fp16.h>

#include "ephdc_internal.cuh"

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t* status,
                                          uint32_t code) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1ll << 31)) {
      atomicCAS(status, 0u, code);
      return false;
    }
  }
  return true;
}
// shared-memory descriptor, K-major without swizzle: 8-row x 16-byte core matrices,
// LBO = byte stride between core matrices along K, SBO = along M/N; version 1
__device__ __forceinline__ uint64_t sdesc_noswz(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
template <uint32_t IDESC>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool ok) {
  const uint32_t d = smem_u32(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(BYTES),
               "r"(ok ? BYTES : 0));
}
// byte u of x and of y as the two fp16 halves (exact integers 0..255): the bytes land
// in the mantissas of 1024.0 (0x6400), and 1024 is subtracted again
__device__ __forceinline__ uint32_t digit_pair(uint32_t x, uint32_t y, uint32_t u) {
  const uint32_t t = __byte_perm(x, y, u | ((u + 4) << 8));  // bytes [x_u, x_0, y_u, x_0]
  uint32_t h = (t & 0x00FF00FFu) | 0x64006400u;
  __half2 v = *reinterpret_cast<const __half2*>(&h);
  v = __hsub2(v, __halves2half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400)));
  return *reinterpret_cast<const uint32_t*>(&v);
}

}  // namespace

namespace {

// byte offset of element (row r, k) in a K-major, no-swizzle operand tile of K = 16:
// core matrices of 8 rows x 8 halves (128 B), the two K-adjacent cores 128 B apart
// (LBO), consecutive 8-row groups 256 B apart (SBO)
__device__ __forceinline__ uint32_t op_off(uint32_t r, uint32_t k) {
  return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// A row of digit u of group g (g < 32 MT): the 4 digits of a group in one warp's
// 32 TMEM lanes, lane u * 8 + g mod 8, warp quarter (g / 8) mod 4, M tile g / 32
__device__ __forceinline__ uint32_t arow(uint32_t u, uint32_t g) {
  return (g >> 3) * 32 + u * 8 + (g & 7);
}

template <int MT, int OP, int KB>
struct TcCfg {
  static constexpr int GP = 32 * MT;               // groups per CTA: A rows (u, g) = 128 MT
  static constexpr int N = 4 * OP;                 // MMA N: columns (v, o)
  static constexpr int KC = 16;                    // plaintexts per chunk = one MMA K step
  static constexpr int WIN = 16;                   // chunks per exact window (256 plaintexts)
  static constexpr int RING = MT == 1 ? 3 : 4;     // cp.async stages of raw residues
  static constexpr int ROWS = GP + OP;             // raw rows per chunk
  static constexpr int PAD = KB == 2 ? 16 : 4;     // row padding (words): conflict-free reads
  static constexpr int RSTRIDE = KC * KB + PAD;    // words per raw row
  static constexpr int RAW_WORDS = ROWS * RSTRIDE;
  static constexpr int A_BYTES = 4 * GP * KC * 2;  // per coefficient
  static constexpr int B_BYTES = N * KC * 2;
  static constexpr int OPS_BYTES = KB * (A_BYTES + B_BYTES);  // one operand buffer
  // operand buffers in flight (the MMAs of chunk c, issued one iteration after its
  // split, must finish before chunk c + NB reuses the buffer)
  static constexpr int NB = 3;
  static constexpr int TCOLS = KB * MT * N;                   // TMEM columns
  static constexpr uint32_t IDESC =
      (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  static constexpr size_t SMEM =
      1024 + NB * OPS_BYTES + RING * RAW_WORDS * 4 + KB * GP * OP * 4 + 128;
};

template <int MT, int OP, int KB>
__global__ void __launch_bounds__(256, 1) k_mac_tc(DevCtx c, const uint32_t* __restrict__ pt,
                                                   const uint32_t* __restrict__ model,
                                                   uint32_t* __restrict__ out, int G,
                                                   uint32_t* status) {
  using C = TcCfg<MT, OP, KB>;
  constexpr int GP = C::GP, N = C::N, KC = C::KC;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* ops = sm;                                                // [NB][KB][A | B]
  uint32_t* raw = (uint32_t*)(sm + C::NB * C::OPS_BYTES);           // [RING][ROWS][RSTRIDE]
  uint32_t* accs = raw + C::RING * C::RAW_WORDS;                   // [KB][OP][GP], mod q_l
  uint64_t* bars = (uint64_t*)(accs + KB * GP * OP);                // MMA done, per buffer (NB <= 4)
  uint32_t* tslot = (uint32_t*)(bars + 4);
  uint32_t* Wsh = tslot + 2;                                        // 2^(8e) mod q_l, e < 7

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t l = blockIdx.y, k0 = blockIdx.x * KB;
  const int g0 = blockIdx.z * GP;
  const int O = 2 * (int)c.Kp;
  const uint32_t P = c.P, n = c.n, L = c.L;
  const ModP m = c.mq[l];
  const int nch = (int)((P + KC - 1) / KC);

  for (int i = tid; i < KB * GP * OP; i += blockDim.x) accs[i] = 0;
  if (tid == 0) {
    for (int b = 0; b < C::NB; b++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[b])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tslot)),
                 "n"(C::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;

  // raw residues of chunk ch: rows g (plaintexts of group g0 + g) and GP + o (model
  // output o), each KC plaintexts x KB coefficients; zero outside the batch.  Every
  // thread copies the same (row, plaintext-in-chunk) pieces in every chunk, so their
  // chunk-0 sources and per-chunk strides are set up once.
  constexpr int COPIES = (C::ROWS * KC + 255) / 256;
  const uint32_t* csrc[COPIES];
  size_t cstep[COPIES];
  int cdst[COPIES], cii[COPIES];
  bool crow[COPIES];
#pragma unroll
  for (int q = 0; q < COPIES; q++) {
    const int t = tid + q * 256;
    const int row = t / KC, ii = t - row * KC;
    cii[q] = ii;
    cdst[q] = t < C::ROWS * KC ? row * C::RSTRIDE + ii * KB : -1;
    if (row < GP) {
      const int g = g0 + row;
      crow[q] = g < G;
      csrc[q] = pt + (((size_t)(crow[q] ? g : 0) * P + ii) * L + l) * n + k0;
      cstep[q] = (size_t)KC * L * n;
    } else {
      const int o = row - GP;
      crow[q] = o < O;
      csrc[q] = model + (((size_t)ii * O + (crow[q] ? o : 0)) * L + l) * n + k0;
      cstep[q] = (size_t)KC * O * L * n;
    }
  }
  auto load_raw = [&](int ch, int stage) {
    uint32_t* dst = raw + stage * C::RAW_WORDS;
#pragma unroll
    for (int q = 0; q < COPIES; q++) {
      if (cdst[q] < 0) continue;
      const bool ok = crow[q] && (uint32_t)(ch * KC + cii[q]) < P;
      cp_async<KB * 4>(dst + cdst[q], ok ? csrc[q] + (size_t)ch * cstep[q] : csrc[q], ok);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  // raw stage -> fp16 digit operand tiles of every coefficient (buffer `buf`)
  auto transform = [&](int stage, int buf) {
    const uint32_t* rs = raw + stage * C::RAW_WORDS;
    uint8_t* ob = ops + buf * C::OPS_BYTES;
    const int glo = lane >> 2, kp = lane & 3;
    constexpr int AITEMS = (GP / 8) * 2, ITEMS = AITEMS + (OP / 8) * 2;
    for (int it = warp; it < ITEMS; it += blockDim.x / 32) {
      const bool isA = it < AITEMS;
      const int jt = isA ? it : it - AITEMS;
      const int hi = jt >> 1, cc = jt & 1;
      const int rr = hi * 8 + glo;                 // group g or output o
      const int ii = cc * 8 + 2 * kp;              // K pair (ii, ii + 1)
      const uint32_t* w = rs + (isA ? rr : GP + rr) * C::RSTRIDE + ii * KB;
      uint32_t x[KB], y[KB];
      if (KB == 4) {
        const uint4 a = *reinterpret_cast<const uint4*>(w);
        const uint4 b = *reinterpret_cast<const uint4*>(w + 4);
        x[0] = a.x; x[1 % KB] = a.y; x[2 % KB] = a.z; x[3 % KB] = a.w;
        y[0] = b.x; y[1 % KB] = b.y; y[2 % KB] = b.z; y[3 % KB] = b.w;
      } else {
        const uint4 a = *reinterpret_cast<const uint4*>(w);  // (x0, x1, y0, y1)
        x[0] = a.x; x[1 % KB] = a.y; y[0] = a.z; y[1 % KB] = a.w;
      }
#pragma unroll
      for (int j = 0; j < KB; j++) {
        uint8_t* tile = ob + j * (C::A_BYTES + C::B_BYTES) + (isA ? 0 : C::A_BYTES);
#pragma unroll
        for (int u = 0; u < 4; u++)
          *reinterpret_cast<uint32_t*>(tile + op_off(isA ? arow(u, rr) : u * OP + rr, ii)) =
              digit_pair(x[j], y[j], u);
      }
    }
  };

  if (tid == 0) {
    uint32_t w = 1;
    for (int e = 0; e < 7; e++, w = mulm(w, 256u, m)) Wsh[e] = w;
  }

  for (int s = 0; s < C::RING - 1; s++) {
    if (s < nch) load_raw(s, s);
    else asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  // window read-out: warp (mt, q) reads TMEM lanes 32 q of M tile mt, i.e. groups
  // (4 mt + q) * 8 + lane % 8 with digit u = lane / 8, and all N columns (v, o)
  auto readout = [&]() {
    if (warp >= 4 * MT) return;
    const int mt = warp >> 2, q = warp & 3;
    const int u = lane >> 3, g = (mt * 4 + q) * 8 + (lane & 7);
#pragma unroll 1
    for (int j = 0; j < KB; j++) {
#pragma unroll 1
      for (int oh = 0; oh < OP; oh += 16) {  // 16 outputs at a time
        uint64_t t[16];
#pragma unroll
        for (int e = 0; e < 16; e++) t[e] = 0;
#pragma unroll
        for (int vv = 0; vv < 4; vv++) {
          uint32_t v[16];
          tc_ld16(tmem + ((uint32_t)(32 * q) << 16) + (j * MT + mt) * N + vv * OP + oh, v);
          const uint64_t w = Wsh[u + vv];
          // S_uv < 2^24 and 2^(8(u+v)) mod q < 2^30: 16 products per output < 2^58
#pragma unroll
          for (int e = 0; e < 16; e++)
            t[e] += (uint64_t)__float2uint_rz(__uint_as_float(v[e])) * w;
        }
#pragma unroll
        for (int e = 0; e < 16; e++) {
          t[e] += __shfl_xor_sync(0xffffffffu, t[e], 8);
          t[e] += __shfl_xor_sync(0xffffffffu, t[e], 16);
        }
        if (u == 0 && g0 + g < G) {
          uint32_t* a = accs + (size_t)j * OP * GP + g;
#pragma unroll
          for (int e = 0; e < 16; e++)
            if (oh + e < O) a[(oh + e) * GP] = red64(t[e] + a[(oh + e) * GP], m.p, m.mu);
        }
      }
    }
  };

  // One block barrier per chunk: at the top of iteration ch every thread's copies of
  // chunk ch have landed and every operand tile of chunk ch - 1 is written, so thread
  // 0 issues the MMAs of chunk ch - 1 while the block loads and splits chunk ch.  An
  // operand buffer is reused NB chunks later, after each thread has seen the MMAs
  // that read it complete (every chunk's completion is awaited in order, so the
  // mbarrier parity is never more than one phase ahead).
  bool alive = true;
  for (int ch = 0; ch <= nch; ch++) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(C::RING - 2) : "memory");
    alive = __syncthreads_and(alive);
    const int pc = ch - 1;
    if (pc >= 0 && tid == 0 && alive) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t ob = smem_u32(ops + (pc % C::NB) * C::OPS_BYTES);
#pragma unroll
      for (int j = 0; j < KB; j++) {
        const uint32_t a0 = ob + j * (C::A_BYTES + C::B_BYTES), b0 = a0 + C::A_BYTES;
        const uint64_t bd = sdesc_noswz(b0, 128, 256);
#pragma unroll
        for (int mt = 0; mt < MT; mt++)
          tc_mma<C::IDESC>(tmem + (j * MT + mt) * N, sdesc_noswz(a0 + mt * 4096, 128, 256), bd,
                           (pc % C::WIN) != 0);
      }
      tc_commit(smem_u32(&bars[pc % C::NB]));
    }
    if (pc >= 0 && ((pc % C::WIN) == C::WIN - 1 || pc == nch - 1)) {
      // window complete: every S_uv of its plaintexts is in TMEM
      const bool ok =
          alive && mbar_wait(smem_u32(&bars[pc % C::NB]), (pc / C::NB) & 1, status, 12);
      alive = __syncthreads_and(ok);
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (alive) readout();
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    }
    if (ch == nch) break;
    {  // raw stage of chunk ch - 1 is free: load chunk ch + RING - 1 into it
      const int nx = ch + C::RING - 1;
      if (nx < nch) load_raw(nx, nx % C::RING);
      else asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    if (ch >= C::NB && alive &&
        !mbar_wait(smem_u32(&bars[ch % C::NB]), ((ch - C::NB) / C::NB) & 1, status, 11))
      alive = false;
    if (alive) transform(ch % C::RING, ch % C::NB);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();
  for (int idx = tid; idx < KB * GP * OP; idx += blockDim.x) {
    const int j = idx % KB, rest = idx / KB;
    const int o = rest % OP, g = rest / OP;
    if (g0 + g < G && o < O)
      out[(((size_t)(g0 + g) * O + o) * L + l) * n + k0 + j] = accs[(j * OP + o) * GP + g];
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "n"(C::TCOLS)
                 : "memory");
}

template <int MT, int OP, int KB>
cudaError_t run_mac_tc(const DevCtx& c, const uint32_t* pt, int G, const uint32_t* model,
                       uint32_t* acc, cudaStream_t st) {
  using C = TcCfg<MT, OP, KB>;
  cudaError_t e = cudaFuncSetAttribute(k_mac_tc<MT, OP, KB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(c.n / KB, c.L, (G + C::GP - 1) / C::GP);
  k_mac_tc<MT, OP, KB><<<grid, 256, C::SMEM, st>>>(c, pt, model, acc, G, c.status);
  return cudaGetLastError();
}

}  // namespace

namespace ephdc {

cudaError_t launch_mac_tc(const DevCtx& c, const uint32_t* pt, int G, const uint32_t* model,
                          uint32_t* acc, cudaStream_t st) {
  const int O = 2 * (int)c.Kp;
  if (O > 32) return cudaErrorNotSupported;
  const bool two = G > 32;  // 64 groups per CTA (two M tiles) beyond 32 groups
  if (O <= 16) return two ? run_mac_tc<2, 16, 4>(c, pt, G, model, acc, st)
                          : run_mac_tc<1, 16, 4>(c, pt, G, model, acc, st);
  return two ? run_mac_tc<2, 32, 2>(c, pt, G, model, acc, st)
             : run_mac_tc<1, 32, 2>(c, pt, G, model, acc, st);
}

}  // namespace ephdc
