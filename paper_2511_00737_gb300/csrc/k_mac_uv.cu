// Dense multiply-accumulate of many groups on the tensor cores as one outer product of
// signed digits (the batch x classes contraction of Sec. 4.1's HE compute when many
// query groups share the model):
//   Acc_k[g][o] = sum_i Pt_k[g][i] * C_k[i][o]  (mod q_l)   for every coefficient k.
//
// Both residues are written in balanced base 256, a = sum_u d_u 2^(8u) and
// c = sum_v e_v 2^(8v) with d_u, e_v in [-128, 127] (the bytes of a + 0x80808080, each
// less 128), so  a c = sum_{u,v} 2^(8(u+v)) d_u e_v.  One MMA per coefficient and 16
// plaintexts computes every digit product at once: A holds the model digits, rows
// (o, v) = 4 o + v (M = 128), B the plaintext digits, rows (u, g) = 16 u + g (N = 64),
// and accumulator element ((v, o), (u, g)) collects sum_i e_v d_u.  Each product is at
// most 2^14 in magnitude, so a window of 1024 plaintexts keeps every fp32 partial sum an
// exact integer within 2^24.  After a window the sums are weighted by 2^(8(u+v)) mod q_l
// and added into accumulators mod q_l.
//
// The model is stored already split (the digit model: for every limb, 8 coefficients
// and 16 plaintexts, the 8 fp16 A operands of 128 rows x 16 columns, 4 KB each, in the
// order mdig_index gives), so a step's model operand is one contiguous 32 KB block
// copied into shared memory by the bulk-copy engine; the CTAs of a cluster
// (consecutive group blocks of the same coefficients) each copy a share of it and
// multicast it to all of them.  Plaintexts stay in the standard layout and arrive as
// 32-byte pieces (8 coefficients of one (group, plaintext) row) through cp.async.
//
// A tile is (limb l, 8 consecutive coefficients, 16 groups; all outputs O <= 32, all
// plaintexts).  Persistent CTAs (clusters) walk their tiles with three kinds of warps:
// 8 splitter warps copy the plaintext pieces NS - 1 steps ahead (across tile
// boundaries), split the current step into digits (B operand, "fullB" mbarrier) and
// read each window out of TMEM; one producer thread bulk-copies the model operand NA
// steps ahead (its expect-tx arrival and the bytes complete "fullA"); one MMA thread
// waits for both, issues the step's 8 MMAs and commits to the digit buffer's local
// "doneB" barrier and to the model buffer's "mfree" barrier in every CTA of the
// cluster (a model buffer is rewritten only after every CTA's MMAs that read it are
// complete).  The 8 accumulators (128 lanes x 64 columns each) fill all 512 TMEM
// columns.  All waits are bounded; a CTA that gave up records the code, stops issuing
// work and still takes part in the cluster barriers.
#include <cuda_fp16.h>

#include "ephdc_internal.cuh"

namespace {

constexpr int SPLITTERS = 256;             // splitter threads (warps 0-7)
constexpr int MMA_WARP = 8, PRODUCER_WARP = 9;
constexpr int THREADS = 320;
constexpr int KB = 8;                       // coefficients per tile
constexpr int GN = 16;                      // groups per tile (N = 4 digits x 16)
constexpr int KC = 16;                      // plaintexts per step = MMA K
constexpr int WINS = 64;                    // steps per exact window (1024 plaintexts)
// model operand of one coefficient: M x 16 fp16 (M = 128 rows: 32 outputs x 4 digits;
// M = 64: 16 outputs x 4 digits, for k/k_in <= 8), and of a step's 8 coefficients
template <int M> __host__ __device__ constexpr int a_tile() { return M * 32; }
template <int M> __host__ __device__ constexpr int a_bytes() { return KB * a_tile<M>(); }
constexpr int B_TILE = 2048;                // plaintext operand of one coefficient: 64 x 16
constexpr int B_BYTES = KB * B_TILE;        // 16 KB per step
constexpr int NA = 4;                       // model operand buffers (bulk-copy lookahead)
constexpr int NB = 2;                       // plaintext digit operand buffers
constexpr int RAW_STEP = GN * KC * 32;      // 8 KB of 32-byte plaintext pieces per step
constexpr int NS = 4;                       // cp.async ring stages
constexpr int TCOLS = 512;
// kind::f16 instruction descriptor: D = f32, A = B = f16, both K-major, N = 64, M
template <int M>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
template <int M>
constexpr size_t smem_bytes() {
  return 1024 + NA * (size_t)a_bytes<M>() + NB * B_BYTES + NS * RAW_STEP + 256;
}
constexpr long long WAIT_LIMIT = 1ll << 29;  // cycles (about a quarter of a second)
static_assert(smem_bytes<128>() <= 232448, "shared memory per CTA");

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
// bounded wait: gives up after WAIT_LIMIT cycles and records `code`
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t* status,
                                          uint32_t code) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_LIMIT) {
      atomicCAS(status, 0u, code);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
// shared-memory descriptor, K-major without swizzle (LBO = 128, SBO = 256), version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(256 >> 4) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc,
                                       uint32_t id) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
      : "memory");
}
// arrive on the mbarrier at the same offset in every CTA of `mask` when the MMAs
// issued so far are complete
__device__ __forceinline__ void tc_commit_mc(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;\n" ::"r"(bar),
      "h"(mask)
      : "memory");
}
// 64 columns of this warp's 32 TMEM lanes into registers, load and wait in one
// statement (so that no use of the registers can be scheduled before the wait)
__device__ __forceinline__ void tc_ld64(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,"
      "%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,"
      "%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
        "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]),
        "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]),
        "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]), "=r"(v[49]),
        "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
        "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]),
        "=r"(v[62]), "=r"(v[63])
      : "r"(taddr)
      : "memory");
}
// 16-byte global -> shared copy, zero-filled when !ok (src must still be a valid address)
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
               "r"(ok ? 16 : 0)
               : "memory");
}
// global -> shared bulk copy of `bytes` into this CTA, or into every CTA of `mask` at
// the same offset; completion counted in bytes on the mbarrier at `bar` of each
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar, uint16_t mask, bool multicast) {
  if (multicast)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
        " [%0], [%1], %2, [%3], %4;\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar), "h"(mask)
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(r));
  return r;
}
// barrier among the 256 splitter threads only
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

}  // namespace

namespace {

// 10 warps: an SM sub-partition holds 3 of them, so at most 168 registers per thread
template <int M>
__global__ void __launch_bounds__(THREADS, 1) k_mac_uv(DevCtx c, const uint32_t* __restrict__ pt,
                                                       const uint16_t* __restrict__ model,
                                                       uint32_t* __restrict__ out, int G,
                                                       uint32_t* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int A_TILE = a_tile<M>(), A_BYTES = a_bytes<M>();
  uint8_t* Areg = sm;                                        // [NA][8][M x 16 fp16]
  uint8_t* Breg = Areg + NA * A_BYTES;                       // [NB][8][64 x 16 fp16]
  uint8_t* ring = Breg + NB * B_BYTES;                       // [NS][16 x 16 pieces of 32 B]
  uint64_t* fullA = (uint64_t*)(ring + NS * RAW_STEP);       // model operand landed
  uint64_t* mfree = fullA + NA;                              // every cluster CTA's MMAs complete
  uint64_t* fullB = mfree + NA;                              // plaintext digits written
  uint64_t* doneB = fullB + NB;                              // this CTA's MMAs complete
  uint64_t* tfree = doneB + NB;                              // window read out of TMEM
  uint32_t* tslot = (uint32_t*)(tfree + 1);
  uint32_t* live0 = tslot + 1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int O = 2 * (int)c.Kp;
  const uint32_t P = c.P, n = c.n, L = c.L, nkt = n / KB;
  const uint32_t S = (P + KC - 1) / KC;  // steps per tile
  const uint32_t CL = cluster_size(), rank = cluster_rank();
  const uint16_t cmask = (uint16_t)((1u << CL) - 1u);
  // cluster tiles: (block of CL consecutive group blocks, 8 coefficients, limb); cluster
  // cid takes cid, cid + NC, ...; this CTA the group block of its rank in each
  const uint32_t GBC = ((G + GN - 1) / GN + CL - 1) / CL, NT = GBC * nkt * L;
  const uint32_t cid = blockIdx.x / CL, NC = gridDim.x / CL;
  const uint32_t T = cid < NT ? (NT - cid + NC - 1) / NC : 0;
  const uint32_t TS = T * S;  // steps of all of this CTA's tiles
  auto tile_of = [&](uint32_t tau, uint32_t& l, uint32_t& k0, int& g0) {
    const uint32_t ct = cid + tau * NC, rest = ct / GBC;
    g0 = (int)(((ct % GBC) * CL + rank) * GN);
    k0 = (rest % nkt) * KB;
    l = rest / nkt;
  };

  if (tid == 0) {
    for (int b = 0; b < NA; b++) {
      mbar_init(smem_u32(&fullA[b]), 1);
      mbar_init(smem_u32(&mfree[b]), CL);
    }
    for (int b = 0; b < NB; b++) {
      mbar_init(smem_u32(&fullB[b]), SPLITTERS);
      mbar_init(smem_u32(&doneB[b]), 1);
    }
    mbar_init(smem_u32(tfree), SPLITTERS);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *live0 = *(volatile uint32_t*)status == 0u;  // a CTA after a recorded failure does no work
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
  cluster_sync();  // every CTA's barriers are initialised before any peer signals them
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  bool alive = *live0 != 0u;

  if (warp == PRODUCER_WARP) {
    // ------------------------------------------------------------ model producer
    if (lane == 0) {
      const uint32_t share = A_BYTES / CL;
      const uint8_t* mbase = reinterpret_cast<const uint8_t*>(model) + rank * share;
      uint32_t tau = 0, s = 0, l = 0, k0 = 0;
      int g0 = 0;
      tile_of(0, l, k0, g0);
      for (uint32_t sg = 0; sg < TS && alive; sg++) {
        const uint32_t b = sg % NA;
        if (sg >= NA && !mbar_wait(smem_u32(&mfree[b]), ((sg / NA) - 1) & 1, status, 21)) {
          alive = false;
          break;
        }
        mbar_arrive_tx(smem_u32(&fullA[b]), A_BYTES);
        bulk_copy(smem_u32(Areg + b * A_BYTES) + rank * share,
                  mbase + (((size_t)l * nkt + k0 / KB) * S + s) * A_BYTES, share,
                  smem_u32(&fullA[b]), cmask, CL > 1);
        if (++s == S) {
          s = 0;
          tile_of(++tau, l, k0, g0);
        }
      }
      // drain: every cluster CTA's MMAs of the last steps (and so every arrival on this
      // CTA's mfree barriers) are complete before the CTA may leave the cluster
      for (uint32_t sg = TS > NA ? TS - NA : 0; sg < TS && alive; sg++)
        if (!mbar_wait(smem_u32(&mfree[sg % NA]), (sg / NA) & 1, status, 22)) alive = false;
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t s = 0, windows = 0;
      for (uint32_t sg = 0; sg < TS && alive; sg++) {
        const uint32_t a = sg % NA, b = sg % NB;
        if (!mbar_wait(smem_u32(&fullA[a]), (sg / NA) & 1, status, 23) ||
            !mbar_wait(smem_u32(&fullB[b]), (sg / NB) & 1, status, 27)) {
          alive = false;
          break;
        }
        const bool first = (s % WINS) == 0;
        if (first) {  // the previous window must have been read out of TMEM
          if (windows > 0 && !mbar_wait(smem_u32(tfree), (windows - 1) & 1, status, 24)) {
            alive = false;
            break;
          }
          windows++;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t a0 = smem_u32(Areg + a * A_BYTES), b0 = smem_u32(Breg + b * B_BYTES);
#pragma unroll
        for (int j = 0; j < KB; j++)
          tc_mma(tmem + (uint32_t)(j * 64), sdesc(a0 + j * A_TILE), sdesc(b0 + j * B_TILE),
                 first ? 0u : 1u, idesc<M>());
        if (CL > 1) tc_commit_mc(smem_u32(&mfree[a]), cmask);
        else tc_commit(smem_u32(&mfree[a]));
        tc_commit(smem_u32(&doneB[b]));
        if (++s == S) s = 0;
      }
    }
  } else {
    // ------------------------------------------------------------ splitter warps
    // copies: 16-byte halves hh of pieces (g, i) (coefficients k0 + 4 hh .. + 3 of group
    // g0 + g, plaintext 16 s + i), two per thread, the two halves of a piece in adjacent
    // threads; slot (i * 16 + g) * 32 with the halves swapped when bit 2 of g is set, so
    // that the split's 4-byte reads of a warp fall in 32 distinct banks.  The copies run
    // NS - 1 steps ahead, across tile boundaries.
    int cg[2], ci[2], chh[2];
    uint32_t dsto[2];
#pragma unroll
    for (int m = 0; m < 2; m++) {
      const int cidx = tid + SPLITTERS * m, pc = cidx >> 1;
      chh[m] = cidx & 1;
      cg[m] = pc & 15;
      ci[m] = pc >> 4;
      dsto[m] = (uint32_t)((ci[m] * 16 + cg[m]) * 32 + 16 * (chh[m] ^ ((cg[m] >> 2) & 1)));
    }
    const size_t pstride = (size_t)L * n;  // words between plaintexts of a group
    uint32_t isg = 0, is = 0, itau = 0;    // next step to copy, its step in its tile, tile
    const uint32_t* isrc[2];
    bool igok[2];
    auto issue_tile = [&]() {
      uint32_t l, k0;
      int g0;
      tile_of(itau, l, k0, g0);
#pragma unroll
      for (int m = 0; m < 2; m++) {
        igok[m] = g0 + cg[m] < G;
        isrc[m] = pt + ((size_t)(igok[m] ? g0 + cg[m] : 0) * P * L + l) * n + k0 + 4 * chh[m];
      }
    };
    issue_tile();
    auto issue = [&]() {
      if (isg < TS && alive) {
        const uint32_t base = smem_u32(ring + (isg % NS) * RAW_STEP);
#pragma unroll
        for (int m = 0; m < 2; m++) {
          const uint32_t i = is * KC + (uint32_t)ci[m];
          const bool ok = igok[m] && i < P;
          cp_async16(base + dsto[m], ok ? isrc[m] + (size_t)i * pstride : pt, ok);
        }
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
      if (isg < TS) {
        isg++;
        if (++is == S) {
          is = 0;
          itau++;
          if (isg < TS) issue_tile();
        }
      }
    };
    // split: coefficient j of pieces (g, 8 h + e), e < 8 -> B rows 16 u + g, columns
    // 8 h .. 8 h + 7 of coefficient j's operand (one 16-byte store per digit u)
    const int sg = (lane & 7) | ((warp & 1) << 3);
    const int sj = ((lane >> 3) & 3) | (((warp >> 2) & 1) << 2);
    const int sh = (warp >> 1) & 1;
    const uint32_t roff = (uint32_t)(sg * 32 + 16 * ((sj >> 2) ^ ((sg >> 2) & 1)) + 4 * (sj & 3));
    auto split = [&](uint32_t step, int buf) {
      const uint8_t* R = ring + (step % NS) * RAW_STEP + roff;
      uint32_t x[8];
#pragma unroll
      for (int e = 0; e < 8; e++)
        x[e] = *reinterpret_cast<const uint32_t*>(R + (8 * sh + e) * 16 * 32) + 0x80808080u;
      uint8_t* Bj = Breg + buf * B_BYTES + sj * B_TILE;
#pragma unroll
      for (int u = 0; u < 4; u++)
        *reinterpret_cast<uint4*>(Bj + mdig_off(16 * u + sg, 8 * sh)) =
            make_uint4(sdigit_pair(x[0], x[1], u), sdigit_pair(x[2], x[3], u),
                       sdigit_pair(x[4], x[5], u), sdigit_pair(x[6], x[7], u));
    };

    // read-out: warp w reads TMEM lanes 32 qv .. 32 qv + 31 (qv = w % 4) of coefficients
    // 4 jj .. 4 jj + 3 (jj = w / 4).  Accumulator row 4 o + v sits in lane 4 o + v
    // (M = 128) or, with M = 64, in lane 32 (r / 16) + r % 16 (lanes 16-31 of each
    // quarter hold none), so lane (o, v) with v = lane % 4 and o = OQ qv + lane / 4 weights
    // the sums of its digit pairs (u, v) by 2^(8(u+v)) mod q_l and the 4 lanes of an
    // output add their partial sums by two exchanges, each lane keeping 4 of the 16
    // groups: g = 8 b0 + 4 b1 + e for lane bits b0, b1 and e < 4.
    constexpr int OQ = M / 16;  // outputs per 32-lane quarter
    const int qv = warp & 3, jj = warp >> 2, dv = lane & 3;
    const int b0 = lane & 1, b1 = (lane >> 1) & 1;
    const int ro = OQ * qv + (lane >> 2), rg = 8 * b0 + 4 * b1;  // this lane's output, groups
    const bool rown = M == 128 || lane < 16;                      // the lane holds accumulators
    // accumulators mod q_l: acc[e2][e] for coefficient 4 jj + e2 and group rg + e
    uint32_t acc[4][4];
#pragma unroll
    for (int e2 = 0; e2 < 4; e2++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[e2][e] = 0;
    uint32_t tl = 0, tk0 = 0;  // the tile being accumulated
    int tg0 = 0;
    ModP m;
    uint32_t W[4];
    uint64_t OFF = 0;
    auto start_tile = [&](uint32_t tau) {
      tile_of(tau, tl, tk0, tg0);
      m = c.mq[tl < L ? tl : 0];
      uint32_t w = 1;
      for (int s = 0; s < dv; s++) w = mulm(w, 256u, m);
      for (int u = 0; u < 4; u++) {
        W[u] = w;
        w = mulm(w, 256u, m);
      }
      // |sum_{u,v} W S| < 16 q 2^24 < 2^58: adding a multiple of q_l above 2^58 keeps it
      // non-negative (and below 2^60)
      OFF = ((1ull << 58) / m.p + 1) * m.p;
    };
    auto readout = [&]() {
#pragma unroll
      for (int e2 = 0; e2 < 4; e2++) {
        uint32_t Sv[64];  // column 16 u + g: digit pair (u, v), group g
        tc_ld64(tmem + ((uint32_t)(32 * qv) << 16) + (uint32_t)((4 * jj + e2) * 64), Sv);
        // exact partial sums in two's complement (lanes without accumulators wrap
        // harmlessly and are never stored)
        uint64_t t[16];
#pragma unroll
        for (int g = 0; g < 16; g++) {
          t[g] = 0;
#pragma unroll
          for (int u = 0; u < 4; u++)
            t[g] += (uint64_t)((int64_t)__float2int_rn(__uint_as_float(Sv[16 * u + g])) *
                               (int64_t)(int32_t)W[u]);
        }
        // sum over the 4 digits v of the output: keep half of the groups, add the
        // partner's half, twice
        uint64_t h[8];
#pragma unroll
        for (int g = 0; g < 8; g++) {
          const uint64_t keep = b0 ? t[g + 8] : t[g], send = b0 ? t[g] : t[g + 8];
          h[g] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
        }
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const uint64_t keep = b1 ? h[e + 4] : h[e], send = b1 ? h[e] : h[e + 4];
          const uint64_t v = keep + __shfl_xor_sync(0xffffffffu, send, 2) + OFF;
          acc[e2][e] = addm(acc[e2][e], red64(v, m.p, m.mu), m.p);
        }
      }
    };

    for (int k = 0; k < NS - 1; k++) issue();
    start_tile(0);
    uint32_t s = 0, tau = 0;
#pragma unroll 1
    for (uint32_t sgl = 0; sgl < TS; sgl++) {
      const int b = (int)(sgl % NB);
      asm volatile("cp.async.wait_group %0;\n" ::"n"(NS - 2) : "memory");
      splitters_sync();  // every thread's pieces of this step have landed
      issue();
      // the buffer's previous MMAs (step sgl - NB) must be done before it is rewritten
      if (sgl >= NB && alive &&
          !mbar_wait(smem_u32(&doneB[b]), ((sgl / NB) - 1) & 1, status, 25))
        alive = false;
      if (alive) split(sgl, b);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_arrive(smem_u32(&fullB[b]));
      if ((s % WINS) == WINS - 1 || s == S - 1) {
        const bool ok = alive && mbar_wait(smem_u32(&doneB[b]), (sgl / NB) & 1, status, 26);
        alive = splitters_and(ok);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (alive) readout();
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        mbar_arrive(smem_u32(tfree));
      }
      if (++s == S) {
        // coefficients 4 jj .. 4 jj + 3 of (group rg + e, output ro): one 16-byte store each
#pragma unroll
        for (int e = 0; e < 4; e++) {
          if (alive && rown && tg0 + rg + e < G && ro < O) {
            uint4* dst = reinterpret_cast<uint4*>(
                out + (((size_t)(tg0 + rg + e) * O + ro) * L + tl) * n + tk0 + 4 * jj);
            *dst = make_uint4(acc[0][e], acc[1][e], acc[2][e], acc[3][e]);
          }
        }
#pragma unroll
        for (int e2 = 0; e2 < 4; e2++)
#pragma unroll
          for (int e = 0; e < 4; e++) acc[e2][e] = 0;
        s = 0;
        if (++tau < T) start_tile(tau);
      }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "n"(TCOLS)
                 : "memory");
  // after a recorded failure some waits were skipped: give copies and commits already
  // issued (by this CTA or a peer) 50 us to land before the CTAs leave the cluster
  if (tid == 0 && *(volatile uint32_t*)status != 0u) {
    const long long t0 = clock64();
    while (clock64() - t0 < 100000ll) __nanosleep(1000);
  }
  __syncwarp();    // the aligned cluster barrier wants the whole warp converged
  cluster_sync();  // no CTA leaves while a peer may still signal or fill it
}

}  // namespace

namespace ephdc {

template <int M>
static cudaError_t launch_uv(const DevCtx& c, const uint32_t* pt, int G, const uint16_t* model,
                             uint32_t* acc, int cluster, cudaStream_t st) {
  constexpr size_t SMEM = smem_bytes<M>();
  cudaError_t e =
      cudaFuncSetAttribute(k_mac_uv<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
  if (e != cudaSuccess) return e;
  // a power of two (each CTA copies a_bytes / cl bytes, a multiple of 16), at most the
  // power of two that covers the group blocks
  const int gb = (G + GN - 1) / GN;
  int cover = 1;
  while (cover < gb) cover *= 2;
  int cl = cluster > 0 ? cluster : 4;
  if (cl & (cl - 1) || cl > 8) return cudaErrorInvalidValue;
  if (cl > cover) cl = cover;
  // persistent: as many clusters as are resident at once, each walking its tiles
  const long long tiles = (long long)((gb + cl - 1) / cl) * (c.n / KB) * c.L;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = SMEM;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((unsigned)cl);
  // resident clusters per device and cluster size, asked once (a host-side query)
  static int resident_cache[64][4];  // per operand height (one instantiation each)
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int ci = cl == 1 ? 0 : cl == 2 ? 1 : cl == 4 ? 2 : 3;
  int resident = dev < 64 ? resident_cache[dev][ci] : 0;
  if (resident < 1) {
    if (cudaOccupancyMaxActiveClusters(&resident, k_mac_uv<M>, &cfg) != cudaSuccess ||
        resident < 1) {
      cudaGetLastError();
      int sms = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      resident = sms / cl > 0 ? sms / cl : 1;
    }
    if (dev < 64) resident_cache[dev][ci] = resident;
  }
  const long long nc = tiles < resident ? tiles : resident;
  cfg.gridDim = dim3((unsigned)(nc * cl));
  return cudaLaunchKernelEx(&cfg, k_mac_uv<M>, c, pt, model, acc, G, c.status);
}

cudaError_t launch_mac_uv(const DevCtx& c, const uint32_t* pt, int G, const uint16_t* model,
                          uint32_t* acc, int cluster, cudaStream_t st) {
  if (2 * (int)c.Kp > 32 || c.n % KB || G < 1) return cudaErrorNotSupported;
  // the digit model's tile height (mdig_rows) is the MMA's M
  return mdig_rows(c.Kp) == 64 ? launch_uv<64>(c, pt, G, model, acc, cluster, st)
                               : launch_uv<128>(c, pt, G, model, acc, cluster, st);
}

}  // namespace ephdc
