// Dense multiply-accumulate of many groups on the tensor cores (the batch x classes
// contraction of Sec. 4.1's HE compute when many query groups share the model):
//   Acc_k[g][o] = sum_i Pt_k[g][i] * C_k[i][o]  (mod q_l)   for every coefficient k.
//
// Exact signed-digit split: a residue a < 2^30 is written in balanced base 256,
// a = sum_{u<4} d_u 2^(8u) with d_u in [-128, 127] (the bytes of a + 0x80808080, each
// less 128), and likewise c = sum_v e_v 2^(8v).  Then
//   sum_i a c = sum_{s=0..6} 2^(8s) S_s,   S_s = sum_i sum_{u+v=s} d_u e_v,
// and every S_s is computed by the tensor cores exactly: digits are fp16 integers,
// products are at most 2^14 in magnitude, at most 4 of them share an (i, s), and a
// window of 256 plaintexts keeps every fp32 partial sum within 2^24.
//
// Shifted operand: the model digits of a coefficient are 4 blocks of 32 rows (one row
// per output o), block v holding digit e_v, with 3 zero blocks before and after.  The
// A operand of plaintext digit u is the 128-row window starting u blocks before digit
// 0 (rows (s, o), s = 0..3) or 4 - u blocks after it (s = 4..7), so one MMA per
// (u, window) with d_u as B (N = 64 groups) adds exactly the products with u + v = s
// into accumulator row (s, o).  7 MMAs of M = 128, N = 64, K = 16 per coefficient and
// 16 plaintexts; the accumulators of one coefficient take 128 TMEM columns, so a CTA
// holds 4 coefficients (all 512 columns) and every global read is a 16-byte piece.
//
// One CTA per tile (limb l, 4 consecutive coefficients, a block of 64 groups; all
// outputs O <= 32, all plaintexts), walked in 16-plaintext steps by two kinds of warps.
// Eight splitter warps copy their 16-byte pieces of the step NS - 1 ahead into a
// shared-memory ring with cp.async, split their pieces of the current step into
// digits (two operand buffers) and arrive on the buffer's "full" mbarrier; one MMA
// warp waits for it, issues the step's 28 MMAs and commits to the buffer's "done"
// mbarrier, which frees the buffer.  After each window the splitter warps read the
// accumulators out of TMEM, weight S_s by 2^(8s) mod q_l, sum over s across warps in
// shared memory, add into accumulators mod q_l held in registers and release TMEM to
// the MMA warp; the tile's last window stores them.  Tiles with neighbouring
// coefficients run side by side and share every 32-byte sector.  All waits are
// bounded.
#include <cuda_fp16.h>

#include "ephdc_internal.cuh"

namespace {

constexpr int SPLITTERS = 256;            // splitter threads (warps 0-7)
constexpr int THREADS = SPLITTERS + 32;    // + the MMA warp
constexpr int KB = 4;                      // coefficients per tile
constexpr int GN = 64;                     // groups per tile = MMA N
constexpr int OR = 32;                     // output rows per digit block (O <= 32)
constexpr int KC = 16;                     // plaintexts per step = MMA K
constexpr int WIN = 16;                    // steps per exact window (256 plaintexts)
constexpr int ZBLK = OR * KC * 2;          // one digit block: 32 rows x 16 halves = 1 KB
// model digit blocks: 3 zero blocks, then per coefficient 4 digit blocks and 3 zero
// blocks (the zeros after one coefficient are the zeros before the next)
constexpr int ZBLOCKS = 3 + KB * 7;
__host__ __device__ constexpr int zdigit0(int j) { return 3 + 7 * j; }
constexpr int BT_BYTES = GN * KC * 2;      // plaintext digit tile, per (coefficient, u)
constexpr int A_REGION = ZBLOCKS * ZBLK;   // 31 KB
constexpr int B_REGION = KB * 4 * BT_BYTES;  // 32 KB
constexpr int OPS_BYTES = A_REGION + B_REGION;
constexpr int NBUF = 2;                    // operand buffers
constexpr int NS = 4;                      // cp.async ring stages of raw pieces
constexpr int RAW_PT = GN * KC * 16;       // 16 KB: pieces (g, i)
constexpr int RAW_BYTES = RAW_PT + KC * OR * 16;  // + 8 KB: pieces (i, o)
constexpr int TCOLS = 512;
// kind::f16 instruction descriptor: D = f32, A = B = f16, both K-major, N = 64, M = 128
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(GN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr size_t SMEM = 1024 + NBUF * OPS_BYTES + NS * RAW_BYTES + 128;
static_assert(B_REGION >= 4 * GN * OR * 4, "the read-out staging lives in a B region");
static_assert(SMEM <= 232448, "shared memory per CTA");

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
// bounded wait: gives up after ~2^31 cycles (about a second) and records `code`
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
// load and wait in one statement, so that no use of the registers can be scheduled
// before the wait
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
// 16-byte global -> shared copy, zero-filled when !ok (src must still be a valid address)
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
               "r"(ok ? 16 : 0)
               : "memory");
}
// signed digit u of two residues as the two fp16 halves: xb, yb are the residues plus
// 0x80808080, so byte u is d_u + 128; the byte lands in the mantissa of 1024.0
// (0x6400) and 1152 = 1024 + 128 is subtracted, all exactly
__device__ __forceinline__ uint32_t sdigit_pair(uint32_t xb, uint32_t yb, uint32_t u) {
  const uint32_t t = __byte_perm(xb, yb, u | ((u + 4) << 8));  // bytes [x_u, x_0, y_u, x_0]
  uint32_t h = (t & 0x00FF00FFu) | 0x64006400u;
  __half2 v = *reinterpret_cast<const __half2*>(&h);
  v = __hsub2(v, __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480)));
  return *reinterpret_cast<const uint32_t*>(&v);
}
// byte offset of element (row r, k) in a K-major, no-swizzle operand tile of K = 16:
// core matrices of 8 rows x 8 halves (128 B), the two K-adjacent cores 128 B apart
// (LBO), consecutive 8-row groups 256 B apart (SBO)
__device__ __forceinline__ uint32_t op_off(uint32_t r, uint32_t k) {
  return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint32_t comp(const uint4& v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

}  // namespace


namespace {

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
// barrier among the 256 splitter threads only (the MMA warp runs on)
__device__ __forceinline__ void splitters_sync() {
  asm volatile("bar.sync 1, %0;\n" ::"n"(SPLITTERS) : "memory");
}
// the same barrier, returning whether every splitter thread passed true
__device__ __forceinline__ bool splitters_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n barrier.red.and.pred p, 1, %2, q;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(SPLITTERS)
      : "memory");
  return r != 0;
}

// 9 warps: an SM sub-partition holds 3 of them, so at most 168 registers per thread
__global__ void __launch_bounds__(THREADS, 1) k_mac_tc(DevCtx c, const uint32_t* __restrict__ pt,
                                                       const uint32_t* __restrict__ model,
                                                       uint32_t* __restrict__ out, int G,
                                                       uint32_t* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* ops = sm;                                         // [NBUF][A_REGION | B_REGION]
  uint8_t* ring = sm + NBUF * OPS_BYTES;                     // [NS][RAW_BYTES]
  uint64_t* full = (uint64_t*)(ring + NS * RAW_BYTES);       // operands written, per buffer
  uint64_t* done = full + NBUF;                              // MMAs complete, per buffer
  uint64_t* tfree = done + NBUF;                             // window read out of TMEM
  uint32_t* tslot = (uint32_t*)(tfree + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int O = 2 * (int)c.Kp;
  const uint32_t P = c.P, n = c.n, L = c.L;
  const uint32_t l = blockIdx.y, k0 = blockIdx.x * KB;
  const int g0 = blockIdx.z * GN;
  const int steps = (int)((P + KC - 1) / KC);

  {  // zero both operand buffers (the zero digit blocks of the model operand stay zero)
    uint4* z = reinterpret_cast<uint4*>(ops);
    for (int i = tid; i < NBUF * OPS_BYTES / 16; i += THREADS) z[i] = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    for (int b = 0; b < NBUF; b++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&full[b])),
                   "r"(SPLITTERS));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&done[b])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(tfree)),
                 "r"(SPLITTERS));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tslot)),
                 "n"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == SPLITTERS / 32) {
    // ------------------------------------------------------------ MMA warp
    if (lane == 0) {
      for (int s = 0; s < steps; s++) {
        const int b = s & 1;
        if (!mbar_wait(smem_u32(&full[b]), (s >> 1) & 1, status, 15)) break;
        const bool first_of_window = (s % WIN) == 0;
        if (first_of_window && s > 0 &&
            !mbar_wait(smem_u32(tfree), ((s / WIN) - 1) & 1, status, 16))
          break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t a0 = smem_u32(ops + b * OPS_BYTES), b0 = a0 + A_REGION;
#pragma unroll
        for (int j = 0; j < KB; j++) {
#pragma unroll
          for (int tile = 0; tile < 2; tile++) {
            const uint32_t d = tmem + (uint32_t)((j * 2 + tile) * GN);
#pragma unroll
            for (int u = tile; u < 4; u++) {
              const uint32_t aa = a0 + (zdigit0(j) + 4 * tile - u) * ZBLK;
              const uint32_t bb = b0 + (j * 4 + u) * BT_BYTES;
              tc_mma(d, sdesc_noswz(aa, 128, 256), sdesc_noswz(bb, 128, 256),
                     (first_of_window && u == tile) ? 0u : 1u);
            }
          }
        }
        tc_commit(smem_u32(&done[b]));
      }
    }
  } else {
    // ------------------------------------------------------------ splitter warps
    // Pieces of a step: plaintext rows (g, i) of group g = tid / 4 and plaintexts
    // 4 (tid % 4) .. + 3; model rows (i, o) of output o = 8 (warp % 4) + lane / 4 and
    // plaintexts 8 (warp / 4) + 2 (lane % 4) .. + 1.  Each piece is the 16 bytes of the
    // tile's 4 coefficients; rows outside the batch are zero-filled.  Every thread reads
    // back only the pieces it copied, so its own cp.async wait orders them.  Plaintext
    // pieces sit i-major in the ring (slot i * 64 + g), so the 16-byte reads of a warp
    // spread over all banks.
    const int pg = tid >> 2, pq = (tid & 3) * 4;
    const int mo = (warp & 3) * 8 + (lane >> 2), mi = (warp >> 2) * 8 + 2 * (lane & 3);
    const bool gok = g0 + pg < G, ook = mo < O;
    const uint32_t gg = gok ? g0 + pg : 0, oo = ook ? mo : 0;
    const uint32_t* pbase = c.layout ? pt + blk_index(n, G, P, gg, 0, l, k0)
                                     : pt + ((size_t)gg * P * L + l) * n + k0;
    const size_t ps = c.layout ? 4 : (size_t)L * n;
    const uint32_t* mbase = c.layout ? model + blk_index(n, P, O, 0, oo, l, k0)
                                     : model + ((size_t)oo * L + l) * n + k0;
    const size_t ms = c.layout ? (size_t)O * 4 : (size_t)O * L * n;
    auto issue = [&](int s) {
      if (s < steps) {
        const uint32_t dst = smem_u32(ring + (s % NS) * RAW_BYTES);
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const uint32_t i = (uint32_t)(s * KC + pq + e);
          const bool ok = gok && i < P;
          cp_async16(dst + ((pq + e) * GN + pg) * 16, ok ? pbase + i * ps : pt, ok);
        }
#pragma unroll
        for (int e = 0; e < 2; e++) {
          const uint32_t i = (uint32_t)(s * KC + mi + e);
          const bool ok = ook && i < P;
          cp_async16(dst + RAW_PT + ((mi + e) * OR + mo) * 16, ok ? mbase + i * ms : model, ok);
        }
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    // this thread's raw pieces of step s -> signed fp16 digits in operand buffer `buf`
    auto split = [&](int s, int buf) {
      const uint8_t* R = ring + (s % NS) * RAW_BYTES;
      uint4 x[4], y[2];
#pragma unroll
      for (int e = 0; e < 4; e++)
        x[e] = *reinterpret_cast<const uint4*>(R + ((pq + e) * GN + pg) * 16);
#pragma unroll
      for (int e = 0; e < 2; e++)
        y[e] = *reinterpret_cast<const uint4*>(R + RAW_PT + ((mi + e) * OR + mo) * 16);
      uint8_t* A = ops + buf * OPS_BYTES;
      uint8_t* B = A + A_REGION;
#pragma unroll
      for (int j = 0; j < KB; j++) {
        const uint32_t x0 = comp(x[0], j) + 0x80808080u, x1 = comp(x[1], j) + 0x80808080u;
        const uint32_t x2 = comp(x[2], j) + 0x80808080u, x3 = comp(x[3], j) + 0x80808080u;
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const uint2 v = make_uint2(sdigit_pair(x0, x1, u), sdigit_pair(x2, x3, u));
          *reinterpret_cast<uint2*>(B + (j * 4 + u) * BT_BYTES + op_off(pg, pq)) = v;
        }
        const uint32_t y0 = comp(y[0], j) + 0x80808080u, y1 = comp(y[1], j) + 0x80808080u;
#pragma unroll
        for (int v = 0; v < 4; v++)
          *reinterpret_cast<uint32_t*>(A + (zdigit0(j) + v) * ZBLK + op_off(mo, mi)) =
              sdigit_pair(y0, y1, v);
      }
    };

    // accumulators mod q_l: pairs idx = tid + 256 r = g * 32 + o (group g, output o)
    // of each coefficient j
    uint32_t acc[KB][8];
#pragma unroll
    for (int j = 0; j < KB; j++)
#pragma unroll
      for (int r = 0; r < 8; r++) acc[j][r] = 0;
    uint32_t* stage = reinterpret_cast<uint32_t*>(ops + A_REGION);  // [4 qd][GN][OR]
    const ModP m = c.mq[l];
    // read-out: warp w reads TMEM lanes 32 (w % 4) + o (rows s = w % 4 and s = 4 + w % 4
    // of output o) for groups 32 (w / 4) .. + 31, weighted by 2^(8s) mod q_l
    const int qd = warp & 3, hf = warp >> 2;
    uint32_t W0 = 1, W1 = 0;
    for (int s = 0; s < qd; s++) W0 = mulm(W0, 256u, m);
    if (qd < 3) {
      W1 = W0;
      for (int s = 0; s < 4; s++) W1 = mulm(W1, 256u, m);
    }
    // |S0 W0 + S1 W1| < 2^55: adding a multiple of q_l above 2^56 keeps it non-negative
    const int64_t OFF = (int64_t)(((1ull << 56) / m.p + 1) * m.p);
    auto readout = [&]() {
#pragma unroll
      for (int j = 0; j < KB; j++) {
#pragma unroll 1
        for (int h = 0; h < 32; h += 16) {  // 16 groups at a time
          uint32_t v0[16], v1[16];
          const uint32_t ta =
              tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(j * 2 * GN + hf * 32 + h);
          tc_ld16(ta, v0);
          tc_ld16(ta + GN, v1);
#pragma unroll
          for (int e = 0; e < 16; e++) {
            const int64_t v = (int64_t)__float2int_rn(__uint_as_float(v0[e])) * W0 +
                              (int64_t)__float2int_rn(__uint_as_float(v1[e])) * W1 + OFF;
            stage[(qd * GN + hf * 32 + h + e) * OR + lane] = red64((uint64_t)v, m.p, m.mu);
          }
        }
        splitters_sync();
#pragma unroll
        for (int r = 0; r < 8; r++) {
          const int idx = tid + SPLITTERS * r;
          const uint64_t t = (uint64_t)acc[j][r] + stage[idx] + stage[GN * OR + idx] +
                             stage[2 * GN * OR + idx] + stage[3 * GN * OR + idx];
          acc[j][r] = red64(t, m.p, m.mu);
        }
        splitters_sync();
      }
    };

    bool alive = true;
    for (int s = 0; s < NS - 1; s++) issue(s);
#pragma unroll 1
    for (int s = 0; s < steps; s++) {
      const int b = s & 1;
      asm volatile("cp.async.wait_group %0;\n" ::"n"(NS - 2) : "memory");
      // the buffer's previous MMAs (step s - 2) must be done before it is rewritten
      if (s >= 2 && alive && !mbar_wait(smem_u32(&done[b]), ((s - 2) >> 1) & 1, status, 13))
        alive = false;
      if (alive) split(s, b);
      issue(s + NS - 1);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_arrive(smem_u32(&full[b]));
      if ((s % WIN) == WIN - 1 || s == steps - 1) {
        const bool ok = alive && mbar_wait(smem_u32(&done[b]), (s >> 1) & 1, status, 14);
        alive = splitters_and(ok);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (alive) readout();
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        mbar_arrive(smem_u32(tfree));
      }
    }
    // the 4 consecutive coefficients of (group, output) as one 16-byte store
#pragma unroll
    for (int r = 0; r < 8; r++) {
      const int g = (tid >> 5) + 8 * r, o = tid & 31;
      if (alive && g0 + g < G && o < O)
        *reinterpret_cast<uint4*>(out + (((size_t)(g0 + g) * O + o) * L + l) * n + k0) =
            make_uint4(acc[0][r], acc[1][r], acc[2][r], acc[3][r]);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "n"(TCOLS)
                 : "memory");
}

}  // namespace

namespace ephdc {

cudaError_t launch_mac_tc(const DevCtx& c, const uint32_t* pt, int G, const uint32_t* model,
                          uint32_t* acc, cudaStream_t st) {
  if (2 * (int)c.Kp > OR || c.n % KB) return cudaErrorNotSupported;
  cudaError_t e =
      cudaFuncSetAttribute(k_mac_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(c.n / KB, c.L, (G + GN - 1) / GN);
  k_mac_tc<<<grid, THREADS, SMEM, st>>>(c, pt, model, acc, G, c.status);
  return cudaGetLastError();
}

}  // namespace ephdc
