// Host side of the EP-HDC CUDA library: parameter derivation, device tables,
// context and scratch management, and the C-ABI entry points declared in
// include/ephdc.h.  Every step of the inference path runs in the kernels of the
// k_*.cu files; this file only validates arguments, derives constants and enqueues
// launches.  Each stage is an NVTX range (header-only NVTX: free unless a profiler
// is attached) and, when profiling is on, a pair of CUDA events.
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ephdc_internal.cuh"

namespace {

// ------------------------------------------------------------------ number theory
uint32_t pw(uint64_t b, uint64_t e, uint32_t m) {
  unsigned __int128 r = 1, x = b % m;
  while (e) {
    if (e & 1) r = (r * x) % m;
    x = (x * x) % m;
    e >>= 1;
  }
  return (uint32_t)r;
}

// Miller-Rabin with the witnesses {2, 7, 61}, exact for all 32-bit inputs.
bool prime32(uint32_t v) {
  if (v < 2) return false;
  for (uint32_t sp : {2u, 3u, 5u, 7u, 11u, 13u, 61u})
    if (v % sp == 0) return v == sp;
  uint32_t d = v - 1, s = 0;
  while (!(d & 1)) d >>= 1, s++;
  for (uint32_t a : {2u, 7u, 61u}) {
    uint64_t x = pw(a, d, v);
    if (x == 1 || x == v - 1) continue;
    bool witness = true;
    for (uint32_t i = 1; i < s && witness; i++) {
      x = (x * x) % v;
      if (x == v - 1) witness = false;
    }
    if (witness) return false;
  }
  return true;
}

uint32_t brv_host(uint32_t v, uint32_t bits) {
  uint32_t r = 0;
  for (uint32_t i = 0; i < bits; i++) r |= ((v >> i) & 1u) << (bits - 1 - i);
  return r;
}

// primitive 2n-th root: x^((p-1)/2n) for the least quadratic non-residue x
uint32_t root2n(uint32_t p, uint32_t n) {
  uint32_t x = 2;
  while (pw(x, (p - 1) / 2, p) != p - 1) x++;
  return pw(x, (p - 1) / (2ull * n), p);
}

uint32_t shoup(uint32_t w, uint32_t p) { return (uint32_t)(((uint64_t)w << 32) / p); }

// little-endian multi-word helpers (host)
void bmul(uint32_t* a, uint32_t m) {
  uint64_t c = 0;
  for (int i = 0; i < EPHDC_BIGW; i++) {
    uint64_t v = (uint64_t)a[i] * m + c;
    a[i] = (uint32_t)v;
    c = v >> 32;
  }
}
uint32_t bdiv(uint32_t* a, uint32_t d) {  // a /= d, returns remainder
  uint64_t r = 0;
  for (int i = EPHDC_BIGW - 1; i >= 0; i--) {
    uint64_t cur = (r << 32) | a[i];
    a[i] = (uint32_t)(cur / d);
    r = cur % d;
  }
  return (uint32_t)r;
}
uint32_t bmod(const uint32_t* a, uint32_t d) {
  uint64_t r = 0;
  for (int i = EPHDC_BIGW - 1; i >= 0; i--) r = ((r << 32) | a[i]) % d;
  return (uint32_t)r;
}

thread_local std::string g_create_error;

}  // namespace

// ------------------------------------------------------------------ context
struct ephdc_ctx {
  ephdc_params prm;
  DevCtx dc;
  int device = 0;
  std::string err;
  // device allocations owned by the context
  void* tables = nullptr;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  int G_max = 0, splits = 1;
  // scratch sub-buffers
  int8_t* H = nullptr;
  uint32_t* pt = nullptr;
  uint32_t* partial = nullptr;
  uint32_t* acc = nullptr;
  uint32_t* tmp = nullptr;
  uint32_t* digits = nullptr;
  // per-stage device timing (ephdc_profile_enable / ephdc_profile_read)
  struct Rec {
    int stage;
    cudaEvent_t a, b;
  };
  bool prof = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  uint64_t launches = 0;
  // MAC schedule (autotuner knobs): mode 0 = automatic, 1 = streaming (split over
  // plaintext ranges), 2 = tiled multi-group
  int mac_mode = 0;
  int mac_min_groups = 4;  // automatic mode: tiled from this many groups on
  // automatic mode: tensor cores from this many groups on (off unless tuned)
  int mac_tc_min_groups = 1 << 30;
  int mac_splits = 0;      // streaming: split count cap (0 = heuristic)
  ephdc::MacTiling tile = {4, 8, 32, 8};
  // digit-outer-product MAC: CTAs per cluster sharing each model block (0 = 4)
  int mac_cluster = 0;
  // ephdc_infer with the tiled MAC: encode and accumulate this many plaintext indices
  // of every group at a time into a reused buffer (0 = the whole pass at once)
  int chunk = 0;
};

static cudaEvent_t take_event(ephdc_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// RAII bracket: records an event pair around one stage on the call's stream
const char* const kStageNames[EPHDC_NSTAGES] = {"ephdc.hdc_encode", "ephdc.encode_plain",
                                                "ephdc.mac", "ephdc.rotate", "ephdc.export",
                                                "ephdc.encrypt_queries"};

struct StageTimer {
  ephdc_ctx* c;
  cudaStream_t st;
  ephdc_ctx::Rec r{};
  StageTimer(ephdc_ctx* c_, int stage, cudaStream_t st_, uint64_t nlaunch) : c(c_), st(st_) {
    c->launches += nlaunch;
    nvtxRangePushA(kStageNames[stage]);
    if (!c->prof) return;
    r.stage = stage;
    r.a = take_event(c);
    r.b = take_event(c);
    cudaEventRecord(r.a, st);
  }
  ~StageTimer() {
    nvtxRangePop();
    if (!c->prof) return;
    cudaEventRecord(r.b, st);
    c->recs.push_back(r);
  }
};

static ephdc_status fail(ephdc_ctx* c, ephdc_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_create_error = buf;
  return s;
}

static ephdc_status cuda_status(ephdc_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return EPHDC_OK;
  return fail(c, EPHDC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static uint32_t groups_for(const ephdc_ctx* c, int32_t B) {
  return (uint32_t)((B + c->dc.cap - 1) / c->dc.cap);
}

static int mac_splits(const DevCtx& dc, int G) {
  // enough (limb, quad, split) threads to fill every SM a few times over
  long per_split = (long)dc.L * (dc.n / 4) * G;
  long want = 152L * 2048;
  long s = (want + per_split - 1) / per_split;
  if (s < 1) s = 1;
  if (s > (long)dc.P) s = dc.P;
  if (s > 64) s = 64;
  return (int)s;
}

extern "C" {

ephdc_status ephdc_ctx_create(const ephdc_params* p, ephdc_ctx** out) {
  if (!out) return fail(nullptr, EPHDC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!p) return fail(nullptr, EPHDC_EINVAL, "params is NULL");
  const uint32_t n = p->n;
  if (n < 1024 || n > 16384 || (n & (n - 1)))
    return fail(nullptr, EPHDC_EINVAL, "n must be a power of two in [1024, 16384], got %u", n);
  if (p->L < 2 || p->L > EPHDC_MAXL)
    return fail(nullptr, EPHDC_EINVAL, "L must be in [2, %d], got %u", EPHDC_MAXL, p->L);
  if (p->k < 1 || p->k_in < 1 || p->k % p->k_in)
    return fail(nullptr, EPHDC_EINVAL, "k_in must divide k (k=%u, k_in=%u)", p->k, p->k_in);
  if (p->r < 1 || (p->r & (p->r - 1)) || p->r > n / (2 * p->k_in))
    return fail(nullptr, EPHDC_EINVAL, "r must be a power of two <= n/(2 k_in), got %u", p->r);
  if (p->D < 1) return fail(nullptr, EPHDC_EINVAL, "D must be positive");
  if (p->F < 16 || p->F % 16 || p->F > 65536)
    return fail(nullptr, EPHDC_EINVAL, "F must be a multiple of 16 in [16, 65536]");
  if (p->hv_bits < 2 || p->hv_bits > 8) return fail(nullptr, EPHDC_EINVAL, "hv_bits must be in [2, 8]");
  if (p->shift < 0 || p->shift > 30) return fail(nullptr, EPHDC_EINVAL, "shift must be in [0, 30]");
  if (p->max_batch < 1) return fail(nullptr, EPHDC_EINVAL, "max_batch must be positive");
  if (!(p->sigma > 0.0 && p->sigma < 100.0)) return fail(nullptr, EPHDC_EINVAL, "sigma out of range");
  const uint32_t t = p->t ? p->t : EPHDC_T_DEFAULT;
  if (t >= (1u << 30) || t % (2 * n) != 1 || !prime32(t))
    return fail(nullptr, EPHDC_EINVAL,
                "t must be a prime = 1 (mod 2n) below 2^30, got %u", t);
  const uint32_t pbits = p->prime_bits ? p->prime_bits : 30;
  if (pbits < 20 || pbits > 30)
    return fail(nullptr, EPHDC_EINVAL, "prime_bits must be in [20, 30], got %u", pbits);
  const uint32_t sgroup = p->scale_group ? p->scale_group : 512;
  if (p->scale_shift > 30)
    return fail(nullptr, EPHDC_EINVAL, "scale_shift must be in [0, 30], got %u", p->scale_shift);

  ephdc_ctx* c = new ephdc_ctx();
  c->prm = *p;
  DevCtx& d = c->dc;
  memset(&d, 0, sizeof d);
  d.n = n;
  d.logn = 0;
  while ((1u << d.logn) < n) d.logn++;
  d.L = p->L; d.k = p->k; d.k_in = p->k_in; d.Kp = p->k / p->k_in; d.r = p->r;
  d.logr = 0;
  while ((1u << d.logr) < p->r) d.logr++;
  d.W = n / (2 * p->r);
  d.cap_row = d.W / p->k_in;
  d.cap = 2 * d.cap_row;
  d.P = (p->D + p->r - 1) / p->r;
  d.D = p->D; d.F = p->F; d.bits = p->hv_bits; d.shift = p->shift;

  d.t = t;
  // the L largest primes q < 2^prime_bits with q = 1 (mod 2n)
  std::vector<uint32_t> q;
  for (uint64_t j = 1; q.size() < p->L; j++) {
    uint64_t cand = (1ull << pbits) - j * 2ull * n + 1;
    if (cand < (1ull << (pbits - 1))) {
      delete c;
      return fail(nullptr, EPHDC_EINVAL, "not enough NTT primes");
    }
    if (prime32((uint32_t)cand)) q.push_back((uint32_t)cand);
  }

  // the centred lift of plaintext coefficients (|v| <= t/2) into Z_{q_l} and the
  // scaled-message arithmetic take t below every RNS prime
  if (t >= q.back()) {
    delete c;
    return fail(nullptr, EPHDC_EINVAL, "t = %u must be below the smallest RNS prime %u", t,
                q.back());
  }
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return fail(nullptr, EPHDC_ECUDA, "no CUDA device");
  }

  // tables: twiddles for L primes + t (2 x n uint2 each), slot maps, Galois elements
  const int nm = p->L + 1;
  size_t tw_bytes = (size_t)nm * 4 * n * sizeof(uint2);  // tw, itw, twl, itwl
  // slot2pos, pos2slot, scatter, and the 256 scaled slot values
  size_t map_bytes = (3 * (size_t)n + 256) * sizeof(uint32_t);
  size_t gal_bytes = 64 * sizeof(uint32_t);
  size_t total = align256(tw_bytes) + align256(map_bytes) + align256(gal_bytes);
  std::vector<uint8_t> host(total, 0);
  uint2* htw = (uint2*)host.data();
  uint32_t* hmap = (uint32_t*)(host.data() + align256(tw_bytes));
  uint32_t* hgal = (uint32_t*)(host.data() + align256(tw_bytes) + align256(map_bytes));

  if (cudaMalloc(&c->tables, total) != cudaSuccess) {
    delete c;
    return fail(nullptr, EPHDC_ENOMEM, "cudaMalloc of %zu table bytes failed", total);
  }
  uint2* dtw = (uint2*)c->tables;
  for (int mi = 0; mi < nm; mi++) {
    const uint32_t pm = mi < (int)p->L ? q[mi] : t;
    const uint32_t psi = root2n(pm, n), psi_inv = pw(psi, pm - 2, pm);
    uint2* f = htw + (size_t)mi * 4 * n;
    uint2* b = f + n;
    uint2* fl = b + n;
    uint2* bl = fl + n;
    for (uint32_t k = 0; k < n; k++) {
      uint32_t e = brv_host(k, d.logn);
      uint32_t w = pw(psi, e, pm), wi = pw(psi_inv, e, pm);
      f[k] = make_uint2(w, shoup(w, pm));
      b[k] = make_uint2(wi, shoup(wi, pm));
    }
    // transposed copies for the contiguous 5-stage pass (blocks of 32 elements)
    const uint32_t M0 = n / 32;
    for (uint32_t r = 0; r < 5; r++)
      for (uint32_t u = 0; u < (1u << r); u++)
        for (uint32_t blk = 0; blk < M0; blk++) {
          fl[((1u << r) - 1 + u) * M0 + blk] = f[((M0 + blk) << r) + u];
          bl[((1u << r) - 1 + u) * M0 + blk] = b[((M0 + blk) << r) + u];
        }
    ModP mp;
    mp.p = pm;
    mp.ninv = pw(n, pm - 2, pm);
    mp.ninv_sh = shoup(mp.ninv, pm);
    mp.mu = (uint64_t)(((unsigned __int128)1 << 64) / pm);
    mp.tw = dtw + (size_t)mi * 4 * n;
    mp.itw = mp.tw + n;
    mp.twl = mp.itw + n;
    mp.itwl = mp.twl + n;
    if (mi < (int)p->L) d.mq[mi] = mp;
    else d.mt = mp;
  }
  // slots: slot index rho*(n/2) + col has exponent e = 3^col (rho = 0) or 2n - 3^col
  // (rho = 1); the device position with exponent e is brv((e - 1) / 2)
  uint32_t* s2p = hmap;
  uint32_t* p2s = hmap + n;
  for (uint32_t rho = 0; rho < 2; rho++)
    for (uint32_t col = 0; col < n / 2; col++) {
      uint32_t e = pw(3, col, 2 * n);
      if (rho) e = 2 * n - e;
      uint32_t pos = brv_host((e - 1) / 2, d.logn);
      uint32_t sidx = rho * (n / 2) + col;
      s2p[sidx] = pos;
      p2s[pos] = sidx;
    }
  // scatter[(qidx * r + ch) * k_in + jin] = device position of slot
  // (rho, ch*W + jin*cap_row + qq), qidx = rho*cap_row + qq: where element ch of the
  // chunk of query qidx lands for class jin
  uint32_t* sct = hmap + 2 * n;
  for (uint32_t qidx = 0; qidx < d.cap; qidx++)
    for (uint32_t ch = 0; ch < d.r; ch++)
      for (uint32_t jin = 0; jin < d.k_in; jin++) {
        const uint32_t rho = qidx / d.cap_row, qq = qidx % d.cap_row;
        const uint32_t sidx = rho * (n / 2) + ch * d.W + jin * d.cap_row + qq;
        sct[(qidx * d.r + ch) * d.k_in + jin] = s2p[sidx] + (s2p[sidx] >> 5);  // padded
      }
  // packed slot value of a hypervector byte b: (int8 b mod t) n^-1 mod t
  uint32_t* hsl = hmap + 3 * n;
  for (uint32_t b = 0; b < 256; b++) {
    const int32_t h = (int8_t)(uint8_t)b;
    const uint64_t v = h < 0 ? (uint64_t)(h + (int64_t)t) : (uint64_t)h;
    hsl[b] = (uint32_t)(v * d.mt.ninv % t);
  }
  for (uint32_t j = 0; j < d.logr; j++) hgal[j] = pw(3, (uint64_t)d.W << j, 2 * n);
  d.slot2pos = (const uint32_t*)((uint8_t*)c->tables + align256(tw_bytes));
  d.pos2slot = d.slot2pos + n;
  d.scatter = d.slot2pos + 2 * n;
  d.hslot = d.slot2pos + 3 * n;
  // whole query rows of r bytes fit one vector load when every row chunk is full
  d.pack_rows = (((d.k_in == 1 && (d.r == 8 || d.r == 16)) || (d.k_in == 2 && d.r == 4)) &&
                 d.D % d.r == 0) ? d.r : 0;
  d.galois = (const uint32_t*)((uint8_t*)c->tables + align256(tw_bytes) + align256(map_bytes));
  cudaError_t ce = cudaMemcpy(c->tables, host.data(), total, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    cudaFree(c->tables);
    delete c;
    return fail(nullptr, EPHDC_ECUDA, "table upload: %s", cudaGetErrorString(ce));
  }

  // Q, floor(Q/t) mod q_l, CRT constants
  uint32_t Qw[EPHDC_BIGW] = {1};
  for (uint32_t l = 0; l < p->L; l++) bmul(Qw, q[l]);
  memcpy(d.big_Q, Qw, sizeof Qw);
  uint32_t Qt[EPHDC_BIGW];
  memcpy(Qt, Qw, sizeof Qw);
  d.rt = bdiv(Qt, t);  // Qt = floor(Q / t), d.rt = Q mod t
  uint32_t Qh[EPHDC_BIGW];
  memcpy(Qh, Qw, sizeof Qw);
  bdiv(Qh, 2);
  memcpy(d.big_Qhalf, Qh, sizeof Qh);
  for (uint32_t l = 0; l < p->L; l++) {
    d.delta[l] = bmod(Qt, q[l]);
    uint32_t hat[EPHDC_BIGW] = {1};
    for (uint32_t o = 0; o < p->L; o++)
      if (o != l) bmul(hat, q[o]);
    memcpy(d.big_Qhat[l], hat, sizeof hat);
    d.qhat_inv[l] = pw(bmod(hat, q[l]), q[l] - 2, q[l]);
  }
  // scaling operation: w = centred lift of (2^s)^-1 mod t into each limb
  if (p->scale_shift) {
    d.scale_g = sgroup;
    const uint32_t u = pw((uint32_t)((1ull << p->scale_shift) % t), t - 2, t);
    for (uint32_t l = 0; l < p->L; l++)
      d.scale_w[l] = u <= (t - 1) / 2 ? u : u + q[l] - t;
  }
  // discrete Gaussian table: T[m] = floor(2^64 P(X <= -19 + m)), weights
  // exp(-x^2 / (2 sigma^2)) on [-19, 19]
  {
    double wgt[2 * 19 + 1], tot = 0.0;
    const double den = 2.0 * p->sigma * p->sigma;
    for (int x = -19; x <= 19; x++) {
      double xx = (double)x * (double)x;
      wgt[x + 19] = std::exp(-(xx / den));
    }
    for (int i = 0; i <= 38; i++) tot += wgt[i];
    double cum = 0.0;
    for (int i = 0; i < EPHDC_CDT_LEN; i++) {
      cum += wgt[i];
      d.cdt[i] = (uint64_t)std::ldexp(cum / tot, 64);
    }
  }

  // default tiling of the multi-group MAC: whole ciphertext columns per warp row
  {
    const int O = 2 * (int)d.Kp;
    const int ot = O % 7 == 0 ? 7 : (O % 8 == 0 || O > 8 ? 8 : 4);
    const int wo = (O + ot - 1) / ot;
    int gt = 4, gc = (16 / (wo > 16 ? 16 : wo)) * gt;
    if (gc > 32) gc = 32;
    if (gc < gt) gt = gc = 2;
    c->tile = {gt, ot, gc, 8};
  }

  // scratch for batches up to max_batch
  c->G_max = (int)groups_for(c, (int32_t)p->max_batch);
  c->splits = mac_splits(d, 1);
  const size_t poly = (size_t)n * sizeof(uint32_t);
  const size_t acc_bytes = (size_t)c->G_max * d.Kp * 2 * d.L * poly;
  // split partial sums: the largest splits(G) * G over the batch sizes allowed
  size_t part_groups = 0;
  for (int G = 1; G <= c->G_max; G++) {
    size_t v = (size_t)mac_splits(d, G) * G;
    if (v > part_groups) part_groups = v;
  }
  size_t off = 0;
  size_t oH = off; off += align256((size_t)p->max_batch * p->D);
  size_t opt = off; off += align256((size_t)c->G_max * d.P * d.L * poly);
  size_t opart = off; off += align256(part_groups * d.Kp * 2 * d.L * poly);
  size_t oacc = off; off += align256(acc_bytes);
  size_t otmp = off; off += align256(acc_bytes);
  size_t odig = off; off += align256((size_t)c->G_max * d.Kp * d.L * poly);
  size_t oxh = off; off += align256((size_t)p->max_batch * p->F * 2);
  size_t owh = off; off += align256((size_t)p->D * p->F * 2);
  size_t ost = off; off += 256;
  c->scratch_bytes = off;
  if (cudaMalloc(&c->scratch, off) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->tables);
    delete c;
    return fail(nullptr, EPHDC_ENOMEM, "cudaMalloc of %zu scratch bytes failed", off);
  }
  uint8_t* sb = (uint8_t*)c->scratch;
  c->H = (int8_t*)(sb + oH);
  c->pt = (uint32_t*)(sb + opt);
  c->partial = (uint32_t*)(sb + opart);
  c->acc = (uint32_t*)(sb + oacc);
  c->tmp = (uint32_t*)(sb + otmp);
  c->digits = (uint32_t*)(sb + odig);
  d.xh = (uint16_t*)(sb + oxh);
  d.wh = (uint16_t*)(sb + owh);
  d.status = (uint32_t*)(sb + ost);
  if (cudaMemset(d.status, 0, 256) != cudaSuccess) {
    cudaFree(c->scratch);
    cudaFree(c->tables);
    delete c;
    return fail(nullptr, EPHDC_ECUDA, "status word initialisation failed");
  }
  *out = c;
  return EPHDC_OK;
}

void ephdc_ctx_destroy(ephdc_ctx* c) {
  if (!c) return;
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  if (c->scratch) cudaFree(c->scratch);
  if (c->tables) cudaFree(c->tables);
  delete c;
}

const char* ephdc_last_error(const ephdc_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

uint64_t ephdc_query(const ephdc_ctx* c, const char* w) {
  if (!c || !w) return 0;
  const DevCtx& d = c->dc;
  if (!strcmp(w, "cap")) return d.cap;
  if (!strcmp(w, "P")) return d.P;
  if (!strcmp(w, "Kp")) return d.Kp;
  if (!strcmp(w, "W")) return d.W;
  if (!strcmp(w, "cap_row")) return d.cap_row;
  if (!strcmp(w, "logr")) return d.logr;
  if (!strcmp(w, "t")) return d.t;
  if (!strcmp(w, "splits")) return (uint64_t)c->splits;
  if (!strcmp(w, "scratch_bytes")) return c->scratch_bytes;
  if (w[0] == 'q' && w[1] >= '0' && w[1] <= '7' && w[2] == 0) {
    uint32_t l = (uint32_t)(w[1] - '0');
    return l < d.L ? d.mq[l].p : 0;
  }
  return 0;
}

size_t ephdc_sk_bytes(const ephdc_ctx* c) {
  return c ? (size_t)c->dc.L * c->dc.n * sizeof(uint32_t) : 0;
}
size_t ephdc_galois_key_bytes(const ephdc_ctx* c) {
  return c ? (size_t)c->dc.logr * c->dc.L * c->dc.L * 4 * c->dc.n * sizeof(uint32_t) : 0;
}
size_t ephdc_model_bytes(const ephdc_ctx* c) {
  if (!c) return 0;
  // the digit model: 2 KB (k/k_in <= 8) or 4 KB per (limb, coefficient, 16 plaintexts)
  if (c->dc.mdig) return mdig_bytes(c->dc.n, c->dc.L, c->dc.P, c->dc.Kp);
  return (size_t)c->dc.P * c->dc.Kp * (c->dc.compact ? 1 : 2) * c->dc.L * c->dc.n *
         sizeof(uint32_t);
}
size_t ephdc_plain_bytes(const ephdc_ctx* c, int32_t B) {
  if (!c || B < 1) return 0;
  return (size_t)groups_for(c, B) * c->dc.P * c->dc.L * c->dc.n * sizeof(uint32_t);
}
size_t ephdc_model_seeded_bytes(const ephdc_ctx* c) {
  return c ? (size_t)c->dc.P * c->dc.Kp * c->dc.L * c->dc.n * sizeof(uint32_t) : 0;
}
size_t ephdc_query_ct_bytes(const ephdc_ctx* c, int32_t B) {
  if (!c || B < 1) return 0;
  return (size_t)groups_for(c, B) * c->dc.P * 2 * c->dc.L * c->dc.n * sizeof(uint32_t);
}
size_t ephdc_model_plain_bytes(const ephdc_ctx* c) {
  return c ? (size_t)c->dc.Kp * c->dc.P * c->dc.L * c->dc.n * sizeof(uint32_t) : 0;
}
size_t ephdc_out_ct_bytes(const ephdc_ctx* c, int32_t B) {
  if (!c || B < 1) return 0;
  return (size_t)groups_for(c, B) * c->dc.Kp * 2 * c->dc.L * c->dc.n * sizeof(uint32_t);
}

}  // extern "C"

// ------------------------------------------------------------------ argument checks
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

#define CHECK_CTX(c)                                                \
  do {                                                              \
    if (!(c)) return EPHDC_EINVAL;                                  \
    (c)->err.clear();                                               \
  } while (0)
#define CHECK_PTR(c, ptr, name)                                                   \
  do {                                                                            \
    if (!(ptr)) return fail(c, EPHDC_EINVAL, "%s is NULL", name);                 \
    if (!aligned16(ptr)) return fail(c, EPHDC_EINVAL, "%s is not 16-byte aligned", name); \
  } while (0)
#define CHECK_B(c, B)                                                                  \
  do {                                                                                 \
    if ((B) < 1 || (uint32_t)(B) > (c)->prm.max_batch)                                 \
      return fail(c, (B) < 1 ? EPHDC_EINVAL : EPHDC_ENOMEM,                            \
                  "batch %d outside [1, max_batch=%u]", (int)(B), (c)->prm.max_batch); \
  } while (0)

static ephdc_status launched(ephdc_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) e = cudaGetLastError();
  return cuda_status(c, e, what);
}

static ephdc_status rotate_export(ephdc_ctx* c, int G, const void* gk, uint32_t* out,
                                  cudaStream_t st);

static ephdc_status similarity_impl(ephdc_ctx* c, const uint32_t* pt, int32_t B,
                                    const void* model, const void* gk, uint32_t* out,
                                    cudaStream_t st) {
  const DevCtx& d = c->dc;
  const int G = (int)groups_for(c, B);
  cudaError_t e;
  {
    const bool tc_ok = 2 * d.Kp <= 32 && d.P < 16384;
    // the blocked layout is read by the tensor-core product only, the compact model by
    // the tiled product only (it regenerates c1 while staging the model)
    if (d.layout && (c->mac_mode == 1 || c->mac_mode == 2))
      return fail(c, EPHDC_EUNSUPPORTED, "the blocked layout needs mac_mode 0 or 3");
    if (d.compact && (c->mac_mode == 1 || c->mac_mode == 3))
      return fail(c, EPHDC_EUNSUPPORTED, "the compact model needs mac_mode 0 or 2");
    // the digit model is read by the digit-outer-product product only, which reads
    // nothing else
    if (d.mdig != (c->mac_mode == 4) && !(d.mdig && c->mac_mode == 0))
      return fail(c, EPHDC_EUNSUPPORTED,
                  d.mdig ? "the digit model needs mac_mode 0 or 4"
                         : "mac_mode 4 needs the digit model (knob model_digits)");
    if (d.mdig) {
      {
        StageTimer tm(c, EPHDC_STAGE_MAC, st, 1);
        e = ephdc::launch_mac_uv(d, pt, G, (const uint16_t*)model, c->acc, c->mac_cluster, st);
      }
      if (e != cudaSuccess) return launched(c, e, "ptct_mac");
      return rotate_export(c, G, gk, out, st);
    }
    const bool tc = !d.compact && tc_ok &&
                    (c->mac_mode == 3 || d.layout ||
                     (c->mac_mode == 0 && G >= c->mac_tc_min_groups));
    const bool tiled = !tc && (c->mac_mode == 2 || d.compact ||
                               (c->mac_mode == 0 && G >= c->mac_min_groups));
    StageTimer tm(c, EPHDC_STAGE_MAC, st, tc || tiled ? 1 : (2 * d.Kp + 3) / 4 + 1);
    if ((c->mac_mode == 3 || d.layout) && !tc_ok) {
      e = cudaErrorNotSupported;
    } else if (tc) {
      e = ephdc::launch_mac_tc(d, pt, G, (const uint32_t*)model, c->acc, st);
    } else if (tiled) {
      e = ephdc::launch_mac_tiled(d, pt, G, (const uint32_t*)model, c->acc, c->tile, st);
    } else {
      const int cap = c->mac_splits > 0 && c->mac_splits < c->splits ? c->mac_splits : c->splits;
      e = ephdc::launch_mac(d, pt, G, (const uint32_t*)model, c->partial, cap, c->acc, st);
    }
  }
  if (e != cudaSuccess) return launched(c, e, "ptct_mac");
  return rotate_export(c, G, gk, out, st);
}

// S7 + S8 on the accumulators in c->acc: rotate-and-sum over the r chunks, then the
// inverse NTT of every limb into the coefficient-domain output ciphertexts
static ephdc_status rotate_export(ephdc_ctx* c, int G, const void* gk, uint32_t* out,
                                  cudaStream_t st) {
  const DevCtx& d = c->dc;
  cudaError_t e;
  const int count = G * (int)d.Kp;
  uint32_t* cur = c->acc;
  if (d.logr) {
    {
      StageTimer tm(c, EPHDC_STAGE_ROTATE, st, 2 * d.logr);
      e = ephdc::launch_rotate_sum(d, c->acc, c->tmp, c->digits, count, (const uint32_t*)gk, st);
    }
    if (e != cudaSuccess) return launched(c, e, "rotate_sum");
    if (d.logr & 1) cur = c->tmp;  // ping-pong: odd number of steps ends in tmp
  }
  {
    StageTimer tm(c, EPHDC_STAGE_EXPORT, st, 1);
    e = ephdc::launch_export(d, cur, count, out, st);
  }
  return launched(c, e, "export");
}

extern "C" {

ephdc_status bfv_keygen(ephdc_ctx* c, uint64_t seed, void* sk, void* gk, void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, sk, "sk_dev");
  if (c->dc.logr) CHECK_PTR(c, gk, "gk_dev");
  return launched(c, ephdc::launch_keygen(c->dc, seed, (uint32_t*)sk, (uint32_t*)gk,
                                          (cudaStream_t)stream), "keygen");
}

ephdc_status bfv_encrypt_model(ephdc_ctx* c, const int8_t* classes, const void* sk, uint64_t seed,
                               void* model, void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, classes, "class_hv_dev");
  CHECK_PTR(c, sk, "sk_dev");
  CHECK_PTR(c, model, "model_dev");
  return launched(c, ephdc::launch_encrypt_model(c->dc, classes, (const uint32_t*)sk, seed,
                                                 (uint32_t*)model, (cudaStream_t)stream),
                  "encrypt_model");
}

ephdc_status bfv_decrypt_scores(ephdc_ctx* c, const void* sk, const uint32_t* out_ct, int32_t B,
                                uint32_t* scores, void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, sk, "sk_dev");
  CHECK_PTR(c, out_ct, "out_ct_dev");
  CHECK_PTR(c, scores, "scores_dev");
  CHECK_B(c, B);
  return launched(c, ephdc::launch_decrypt_scores(c->dc, (const uint32_t*)sk, out_ct, B,
                                                  c->digits, scores, (cudaStream_t)stream),
                  "decrypt_scores");
}

ephdc_status hdc_encode(ephdc_ctx* c, const int8_t* X, const int8_t* Wt, int32_t B, int8_t* H,
                        void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, X, "X_dev");
  CHECK_PTR(c, Wt, "Wt_dev");
  CHECK_PTR(c, H, "H_dev");
  CHECK_B(c, B);
  cudaError_t e;
  {
    StageTimer tm(c, EPHDC_STAGE_HDC, (cudaStream_t)stream, 3);  // widen X, widen Wt, GEMM
    e = ephdc::launch_hdc_encode(c->dc, X, Wt, B, H, (cudaStream_t)stream);
  }
  return launched(c, e, "hdc_encode");
}

ephdc_status bfv_encode_plain(ephdc_ctx* c, const int8_t* H, int32_t B, uint32_t* pt,
                              void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, H, "H_dev");
  CHECK_PTR(c, pt, "pt_dev");
  CHECK_B(c, B);
  cudaError_t e;
  {
    StageTimer tm(c, EPHDC_STAGE_ENCODE, (cudaStream_t)stream, c->dc.scale_g ? 2 : 1);
    e = ephdc::launch_encode_plain(c->dc, H, B, pt, (cudaStream_t)stream);
  }
  return launched(c, e, "encode_plain");
}

ephdc_status bfv_ptct_similarity(ephdc_ctx* c, const uint32_t* pt, int32_t B, const void* model,
                                 const void* gk, uint32_t* out, void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, pt, "pt_dev");
  CHECK_PTR(c, model, "model_dev");
  CHECK_PTR(c, out, "out_ct_dev");
  if (c->dc.logr) CHECK_PTR(c, gk, "gk_dev");
  CHECK_B(c, B);
  return similarity_impl(c, pt, B, model, gk, out, (cudaStream_t)stream);
}

ephdc_status bfv_model_to_digits(ephdc_ctx* c, const void* model, void* model_digits,
                                 void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, model, "model_dev");
  CHECK_PTR(c, model_digits, "model_digits_dev");
  if (!c->dc.mdig)
    return fail(c, EPHDC_EUNSUPPORTED, "the destination is a digit model: set model_digits 1");
  return launched(c, ephdc::launch_model_to_digits(c->dc, (const uint32_t*)model,
                                                   (uint16_t*)model_digits, (cudaStream_t)stream),
                  "model_to_digits");
}

// ------------------------------------------------------------------ seeded model message
ephdc_status bfv_model_to_seeded(ephdc_ctx* c, const void* model, uint32_t* seeded,
                                 void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, model, "model_dev");
  CHECK_PTR(c, seeded, "seeded_dev");
  if (c->dc.layout || c->dc.compact || c->dc.mdig)
    return fail(c, EPHDC_EUNSUPPORTED, "the seeded message needs layout 0 and the full model");
  return launched(c, ephdc::launch_model_to_seeded(c->dc, (const uint32_t*)model, seeded,
                                                   (cudaStream_t)stream),
                  "model_to_seeded");
}

ephdc_status bfv_model_from_seeded(ephdc_ctx* c, const uint32_t* seeded, uint64_t seed,
                                   void* model, void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, seeded, "seeded_dev");
  CHECK_PTR(c, model, "model_dev");
  if (c->dc.layout || c->dc.compact || c->dc.mdig)
    return fail(c, EPHDC_EUNSUPPORTED, "the seeded message needs layout 0 and the full model");
  return launched(c, ephdc::launch_model_from_seeded(c->dc, seeded, seed, (uint32_t*)model,
                                                     (cudaStream_t)stream),
                  "model_from_seeded");
}

// ------------------------------------------------------------------ noise growth
ephdc_status ephdc_find_dmax_trial(ephdc_ctx* c, const void* sk, const int8_t* H, int32_t B,
                                   const int8_t* classes, const uint32_t* pt, const void* model,
                                   int32_t* dmax) {
  CHECK_CTX(c);
  CHECK_PTR(c, sk, "sk_dev");
  CHECK_PTR(c, H, "H_dev");
  CHECK_PTR(c, classes, "class_hv_dev");
  CHECK_PTR(c, pt, "pt_dev");
  CHECK_PTR(c, model, "model_dev");
  if (!dmax) return fail(c, EPHDC_EINVAL, "dmax is NULL");
  const DevCtx& d = c->dc;
  if (d.layout || d.compact || d.mdig)
    return fail(c, EPHDC_EUNSUPPORTED, "the noise-growth trial needs layout 0 and the full model");
  if (d.k != 1 || d.k_in != 1 || d.r != 1)
    return fail(c, EPHDC_EUNSUPPORTED, "needs one class and the layout k_in = 1, r = 1");
  if (B < 1 || (uint32_t)B > d.cap || (uint32_t)B > c->prm.max_batch)
    return fail(c, EPHDC_EINVAL, "B must be in [1, min(cap, max_batch)]");
  const int D = (int)d.D;
  const size_t ln = (size_t)d.L * d.n;
  const size_t xw = (size_t)D * ln, tw = (size_t)ephdc::prefix_chunks(d, D) * ln;
  const size_t sw = (size_t)D * d.cap;
  uint8_t* buf = nullptr;
  const size_t bytes = (xw + tw + sw) * sizeof(uint32_t) + 256;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, EPHDC_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
  }
  uint32_t* X = (uint32_t*)buf;
  uint32_t* T = X + xw;
  uint32_t* scores = T + tw;
  int* first = (int*)(scores + sw);
  cudaError_t e = cudaMemcpy(first, &D, sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = ephdc::launch_prefix_phases(d, pt, (const uint32_t*)model, (const uint32_t*)sk, D, X, T, 0);
  if (e == cudaSuccess) e = ephdc::launch_decrypt_phases(d, X, D, D * (int)d.cap, scores, 0);
  if (e == cudaSuccess) e = ephdc::launch_first_wrong(d, H, classes, B, D, scores, first, 0);
  int v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, first, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_status(c, e, "find_dmax_trial");
  *dmax = v;
  return EPHDC_OK;
}

// ------------------------------------------------------------------ server-side variant
ephdc_status bfv_encrypt_queries(ephdc_ctx* c, const int8_t* H, int32_t B, const void* sk,
                                 uint64_t seed, uint32_t* ctq, void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, H, "H_dev");
  CHECK_PTR(c, sk, "sk_dev");
  if (c->dc.layout) return fail(c, EPHDC_EUNSUPPORTED, "the server-side variant needs layout 0");
  CHECK_PTR(c, ctq, "query_ct_dev");
  CHECK_B(c, B);
  cudaError_t e;
  {
    StageTimer tm(c, EPHDC_STAGE_ENCRYPT, (cudaStream_t)stream, 1);
    e = ephdc::launch_encrypt_queries(c->dc, H, B, (const uint32_t*)sk, seed, ctq,
                                      (cudaStream_t)stream);
  }
  return launched(c, e, "encrypt_queries");
}

ephdc_status bfv_encode_model_plain(ephdc_ctx* c, const int8_t* classes, uint32_t* mm,
                                    void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, classes, "class_hv_dev");
  CHECK_PTR(c, mm, "model_plain_dev");
  if (c->dc.layout) return fail(c, EPHDC_EUNSUPPORTED, "the server-side variant needs layout 0");
  return launched(c, ephdc::launch_encode_model_plain(c->dc, classes, mm, (cudaStream_t)stream),
                  "encode_model_plain");
}

ephdc_status bfv_ctpt_similarity(ephdc_ctx* c, const uint32_t* ctq, int32_t B, const uint32_t* mm,
                                 const void* gk, uint32_t* out, void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, ctq, "query_ct_dev");
  CHECK_PTR(c, mm, "model_plain_dev");
  if (c->dc.layout) return fail(c, EPHDC_EUNSUPPORTED, "the server-side variant needs layout 0");
  CHECK_PTR(c, out, "out_ct_dev");
  if (c->dc.logr) CHECK_PTR(c, gk, "gk_dev");
  CHECK_B(c, B);
  cudaStream_t st = (cudaStream_t)stream;
  const int G = (int)groups_for(c, B);
  cudaError_t e;
  {
    StageTimer tm(c, EPHDC_STAGE_MAC, st, (c->dc.Kp + 3) / 4 + 1);
    e = ephdc::launch_ctpt_mac(c->dc, ctq, G, mm, c->partial, c->splits, c->acc, st);
  }
  if (e != cudaSuccess) return launched(c, e, "ctpt_mac");
  return rotate_export(c, G, gk, out, st);
}

ephdc_status ephdc_infer(ephdc_ctx* c, const int8_t* X, const int8_t* Wt, int32_t B,
                         const void* model, const void* gk, uint32_t* out, void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, X, "X_dev");
  CHECK_PTR(c, Wt, "Wt_dev");
  CHECK_PTR(c, model, "model_dev");
  CHECK_PTR(c, out, "out_ct_dev");
  if (c->dc.logr) CHECK_PTR(c, gk, "gk_dev");
  CHECK_B(c, B);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  {
    StageTimer tm(c, EPHDC_STAGE_HDC, st, 3);  // widen X, widen Wt, GEMM
    e = ephdc::launch_hdc_encode(c->dc, X, Wt, B, c->H, st);
  }
  if (e != cudaSuccess) return launched(c, e, "hdc_encode");
  const DevCtx& d = c->dc;
  const int G = (int)groups_for(c, B);
  const bool tiled =
      !d.mdig && (c->mac_mode == 2 || d.compact ||
                  (c->mac_mode == 0 && G >= c->mac_min_groups && G < c->mac_tc_min_groups));
  if (c->chunk > 0 && (uint32_t)c->chunk < d.P && tiled && !d.layout && !d.scale_g) {
    // plaintext-index chunks: each chunk's plaintexts of all G groups are encoded into
    // the start of the plaintext buffer and accumulated from there, so that they could
    // be read back from L2 rather than HBM (on GB300 they still come from DRAM and the
    // chunked pass is slower than the whole pass)
    for (uint32_t i0 = 0; i0 < d.P && e == cudaSuccess; i0 += (uint32_t)c->chunk) {
      const uint32_t ni = d.P - i0 < (uint32_t)c->chunk ? d.P - i0 : (uint32_t)c->chunk;
      {
        StageTimer tm(c, EPHDC_STAGE_ENCODE, st, 1);
        e = ephdc::launch_encode_plain(d, c->H, B, c->pt, st, i0, ni);
      }
      if (e != cudaSuccess) break;
      StageTimer tm(c, EPHDC_STAGE_MAC, st, 1);
      e = ephdc::launch_mac_tiled(d, c->pt, G, (const uint32_t*)model, c->acc, c->tile, st,
                                  (int)ni, (int)i0, (int)ni, i0 > 0);
    }
    if (e != cudaSuccess) return launched(c, e, "chunked encode + mac");
    return rotate_export(c, G, gk, out, st);
  }
  {
    StageTimer tm(c, EPHDC_STAGE_ENCODE, st, c->dc.scale_g ? 2 : 1);
    e = ephdc::launch_encode_plain(c->dc, c->H, B, c->pt, st);
  }
  if (e != cudaSuccess) return launched(c, e, "encode_plain");
  return similarity_impl(c, c->pt, B, model, gk, out, st);
}

ephdc_status ephdc_ct_to_host_coeff(ephdc_ctx* c, const void* ct, int32_t count, uint32_t* host) {
  CHECK_CTX(c);
  CHECK_PTR(c, ct, "ct_dev");
  if (!host || count < 1) return fail(c, EPHDC_EINVAL, "bad host buffer or count");
  const DevCtx& d = c->dc;
  const size_t words = (size_t)count * 2 * d.L * d.n;
  uint32_t* tmp = nullptr;
  if (cudaMalloc(&tmp, words * 4) != cudaSuccess) return fail(c, EPHDC_ENOMEM, "cudaMalloc");
  cudaError_t e = ephdc::launch_to_coeff(d, (const uint32_t*)ct, tmp, count, 2,
                                         (int)(2 * d.L * d.n), (int)d.n, 0, 0);
  if (e == cudaSuccess) e = cudaMemcpy(host, tmp, words * 4, cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  return cuda_status(c, e, "ct_to_host_coeff");
}

ephdc_status ephdc_gk_to_host_coeff(ephdc_ctx* c, const void* gk, uint32_t* host) {
  CHECK_CTX(c);
  const DevCtx& d = c->dc;
  if (!d.logr) return EPHDC_OK;
  CHECK_PTR(c, gk, "gk_dev");
  if (!host) return fail(c, EPHDC_EINVAL, "host is NULL");
  const int count = (int)(d.logr * d.L);
  const size_t words = (size_t)count * 2 * d.L * d.n;
  uint32_t* tmp = nullptr;
  if (cudaMalloc(&tmp, words * 4) != cudaSuccess) return fail(c, EPHDC_ENOMEM, "cudaMalloc");
  cudaError_t e = ephdc::launch_to_coeff(d, (const uint32_t*)gk, tmp, count, 2,
                                         (int)(d.L * 4 * d.n), (int)(4 * d.n), 1, 0);
  if (e == cudaSuccess) e = cudaMemcpy(host, tmp, words * 4, cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  return cuda_status(c, e, "gk_to_host_coeff");
}

ephdc_status ephdc_plain_to_host_coeff(ephdc_ctx* c, const uint32_t* pt, int32_t count,
                                       uint32_t* host) {
  CHECK_CTX(c);
  CHECK_PTR(c, pt, "pt_dev");
  if (!host || count < 1) return fail(c, EPHDC_EINVAL, "bad host buffer or count");
  const DevCtx& d = c->dc;
  if (d.layout && count % d.P)
    return fail(c, EPHDC_EINVAL, "with the blocked layout count must be groups * P");
  const size_t words = (size_t)count * d.L * d.n;
  uint32_t* tmp = nullptr;
  uint32_t* std_pt = nullptr;
  if (cudaMalloc(&tmp, words * 4) != cudaSuccess) return fail(c, EPHDC_ENOMEM, "cudaMalloc");
  cudaError_t e = cudaSuccess;
  if (d.layout) {  // blocked [L][n/4][G][P][4] -> [G][P][L][n]
    e = cudaMalloc(&std_pt, words * 4);
    if (e == cudaSuccess) e = ephdc::launch_unblock(d, pt, std_pt, count / d.P, d.P, 0);
  }
  if (e == cudaSuccess)
    e = ephdc::launch_to_coeff(d, d.layout ? std_pt : pt, tmp, count, 1, (int)(d.L * d.n),
                               (int)d.n, 0, 0);
  if (e == cudaSuccess) e = cudaMemcpy(host, tmp, words * 4, cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  if (std_pt) cudaFree(std_pt);
  return cuda_status(c, e, "plain_to_host_coeff");
}

ephdc_status ephdc_model_to_host_coeff(ephdc_ctx* c, const void* model, uint32_t* host) {
  CHECK_CTX(c);
  CHECK_PTR(c, model, "model_dev");
  if (!host) return fail(c, EPHDC_EINVAL, "host is NULL");
  const DevCtx& d = c->dc;
  const int count = (int)(d.P * d.Kp);
  const size_t words = (size_t)count * 2 * d.L * d.n;
  uint32_t* tmp = nullptr;
  uint32_t* std_model = nullptr;
  if (cudaMalloc(&tmp, words * 4) != cudaSuccess) return fail(c, EPHDC_ENOMEM, "cudaMalloc");
  cudaError_t e = cudaSuccess;
  if (d.layout) {  // blocked [L][n/4][P][O][4] -> [P][O][L][n]
    e = cudaMalloc(&std_model, words * 4);
    if (e == cudaSuccess)
      e = ephdc::launch_unblock(d, (const uint32_t*)model, std_model, d.P, 2 * d.Kp, 0);
  } else if (d.compact) {  // c0 only -> c0 and the regenerated c1
    e = cudaMalloc(&std_model, words * 4);
    if (e == cudaSuccess)
      e = ephdc::launch_expand_compact(d, (const uint32_t*)model, std_model, 0);
  } else if (d.mdig) {  // digits -> residues
    e = cudaMalloc(&std_model, words * 4);
    if (e == cudaSuccess) e = ephdc::launch_undigit(d, (const uint16_t*)model, std_model, 0);
  }
  if (e == cudaSuccess)
    e = ephdc::launch_to_coeff(d, std_model ? std_model : (const uint32_t*)model, tmp, count, 2,
                               (int)(2 * d.L * d.n), (int)d.n, 0, 0);
  if (e == cudaSuccess) e = cudaMemcpy(host, tmp, words * 4, cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  if (std_model) cudaFree(std_model);
  return cuda_status(c, e, "model_to_host_coeff");
}

ephdc_status ephdc_sk_to_host(ephdc_ctx* c, const void* sk, int32_t* host) {
  CHECK_CTX(c);
  CHECK_PTR(c, sk, "sk_dev");
  if (!host) return fail(c, EPHDC_EINVAL, "host is NULL");
  const DevCtx& d = c->dc;
  int32_t* tmp = nullptr;
  uint32_t* work = nullptr;
  if (cudaMalloc(&tmp, d.n * 4) != cudaSuccess) return fail(c, EPHDC_ENOMEM, "cudaMalloc");
  if (cudaMalloc(&work, d.n * 4) != cudaSuccess) {
    cudaFree(tmp);
    return fail(c, EPHDC_ENOMEM, "cudaMalloc");
  }
  cudaError_t e = ephdc::launch_sk_to_coeff(d, (const uint32_t*)sk, tmp, work, 0);
  if (e == cudaSuccess) e = cudaMemcpy(host, tmp, d.n * 4, cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  cudaFree(work);
  return cuda_status(c, e, "sk_to_host");
}

ephdc_status ephdc_ntt_natural(ephdc_ctx* c, uint32_t limb, uint32_t* poly, int32_t count,
                               int inverse, void* stream) {
  CHECK_CTX(c);
  CHECK_PTR(c, poly, "poly_dev");
  if (limb > c->dc.L || count < 1) return fail(c, EPHDC_EINVAL, "bad limb or count");
  return launched(c, ephdc::launch_ntt_natural(c->dc, limb, poly, count, inverse,
                                               (cudaStream_t)stream), "ntt_natural");
}

ephdc_status ephdc_infer_multi(ephdc_ctx* c, const ephdc_request* reqs, int32_t nreq,
                               const int8_t* Wt, const void* model, const void* gk, uint32_t* out,
                               void* stream) {
  CHECK_CTX(c);
  if (!reqs || nreq < 1) return fail(c, EPHDC_EINVAL, "no requests");
  CHECK_PTR(c, Wt, "Wt_dev");
  CHECK_PTR(c, model, "model_dev");
  CHECK_PTR(c, out, "out_ct_dev");
  if (c->dc.logr) CHECK_PTR(c, gk, "gk_dev");
  int64_t total = 0;
  for (int32_t r = 0; r < nreq; r++) {
    if (reqs[r].B < 0) return fail(c, EPHDC_EINVAL, "request %d has a negative batch", r);
    if (reqs[r].B > 0) CHECK_PTR(c, reqs[r].X_dev, "request X_dev");
    total += reqs[r].B;
  }
  if (total < 1) return fail(c, EPHDC_EINVAL, "all requests are empty");
  if (total > (int64_t)c->prm.max_batch)
    return fail(c, EPHDC_ENOMEM, "packed batch %lld exceeds max_batch=%u", (long long)total,
                c->prm.max_batch);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  {
    // one gather per 64 requests, then widen Wt and the GEMM
    StageTimer tm(c, EPHDC_STAGE_HDC, st, (uint64_t)((nreq + 63) / 64) + 2);
    int32_t row = 0;
    for (int32_t r0 = 0; r0 < nreq && e == cudaSuccess; r0 += 64) {
      ephdc::GatherTable t;
      t.count = 0;
      t.off[0] = row;
      for (int32_t r = r0; r < nreq && r < r0 + 64; r++) {
        t.ptr[t.count] = reqs[r].X_dev;
        row += reqs[r].B;
        t.off[++t.count] = row;
      }
      e = ephdc::launch_gather_widen(c->dc, t, st);
    }
    if (e == cudaSuccess) e = ephdc::launch_hdc_encode(c->dc, nullptr, Wt, (int)total, c->H, st);
  }
  if (e != cudaSuccess) return launched(c, e, "hdc_encode");
  {
    StageTimer tm(c, EPHDC_STAGE_ENCODE, st, c->dc.scale_g ? 2 : 1);
    e = ephdc::launch_encode_plain(c->dc, c->H, (int)total, c->pt, st);
  }
  if (e != cudaSuccess) return launched(c, e, "encode_plain");
  return similarity_impl(c, c->pt, (int32_t)total, model, gk, out, st);
}

ephdc_status ephdc_tune_set(ephdc_ctx* c, const char* knob, int64_t v) {
  CHECK_CTX(c);
  if (!knob) return fail(c, EPHDC_EINVAL, "knob is NULL");
  const int O = 2 * (int)c->dc.Kp;
  if (!strcmp(knob, "mac_mode")) {
    if (v < 0 || v > 4) return fail(c, EPHDC_EINVAL, "mac_mode must be 0, 1, 2, 3 or 4");
    if (v >= 3 && O > 32) return fail(c, EPHDC_EUNSUPPORTED, "tensor-core MAC needs k/k_in <= 16");
    c->mac_mode = (int)v;
  } else if (!strcmp(knob, "model_digits")) {
    if (v < 0 || v > 1) return fail(c, EPHDC_EINVAL, "model_digits must be 0 or 1");
    if (v == 1 && O > 32)
      return fail(c, EPHDC_EUNSUPPORTED, "the digit model needs k/k_in <= 16");
    if (v == 1 && (c->dc.layout || c->dc.compact))
      return fail(c, EPHDC_EUNSUPPORTED, "the digit model needs layout 0 and the full model");
    c->dc.mdig = (uint32_t)v;
  } else if (!strcmp(knob, "mac_cluster")) {
    if (v != 0 && v != 1 && v != 2 && v != 4 && v != 8)
      return fail(c, EPHDC_EINVAL, "mac_cluster must be 0, 1, 2, 4 or 8");
    c->mac_cluster = (int)v;
  } else if (!strcmp(knob, "model_seed")) {
    if (v < -1) return fail(c, EPHDC_EINVAL, "model_seed must be -1 (off) or a seed >= 0");
    if (v >= 0 && (c->dc.layout || c->dc.mdig))
      return fail(c, EPHDC_EUNSUPPORTED, "the compact model needs layout 0 and residues");
    c->dc.compact = v >= 0;
    c->dc.model_seed = v >= 0 ? (uint64_t)v : 0;
  } else if (!strcmp(knob, "chunk")) {
    if (v < 0) return fail(c, EPHDC_EINVAL, "chunk must be >= 0");
    c->chunk = (int)v;
  } else if (!strcmp(knob, "layout")) {
    if (v < 0 || v > 1) return fail(c, EPHDC_EINVAL, "layout must be 0 or 1");
    if (v == 1 && O > 32)
      return fail(c, EPHDC_EUNSUPPORTED, "the blocked layout needs k/k_in <= 16");
    if (v == 1 && (c->dc.compact || c->dc.mdig))
      return fail(c, EPHDC_EUNSUPPORTED, "the blocked layout needs the full residue model");
    c->dc.layout = (uint32_t)v;
  } else if (!strcmp(knob, "ntt_plan")) {
    if (v < 0 || v > 2) return fail(c, EPHDC_EINVAL, "ntt_plan must be 0, 1 or 2");
    c->dc.ntt_plan = (int32_t)v;
  } else if (!strcmp(knob, "hdc_mode")) {
    if (v < 0 || v > 4) return fail(c, EPHDC_EINVAL, "hdc_mode must be 0 .. 4");
    c->dc.hdc_mode = (int32_t)v;
  } else if (!strcmp(knob, "mac_tc_min_groups")) {
    if (v < 1) return fail(c, EPHDC_EINVAL, "mac_tc_min_groups must be >= 1");
    c->mac_tc_min_groups = (int)v;
  } else if (!strcmp(knob, "mac_min_groups")) {
    if (v < 1) return fail(c, EPHDC_EINVAL, "mac_min_groups must be >= 1");
    c->mac_min_groups = (int)v;
  } else if (!strcmp(knob, "mac_splits")) {
    if (v < 0) return fail(c, EPHDC_EINVAL, "mac_splits must be >= 0");
    c->mac_splits = (int)v;
  } else if (!strcmp(knob, "mac_tile")) {
    // packed as gt * 1000000 + ot * 10000 + gc * 100 + ic
    ephdc::MacTiling t = {(int)(v / 1000000), (int)(v / 10000 % 100), (int)(v / 100 % 100),
                          (int)(v % 100)};
    const int wo = (O + t.ot - 1) / (t.ot > 0 ? t.ot : 1);
    const bool shape_ok = (t.gt == 2 || t.gt == 4) && (t.ot == 4 || t.ot == 7 || t.ot == 8);
    if (!shape_ok || t.gc < t.gt || t.gc % t.gt || t.gc > 64 || (t.gc / t.gt) * wo > 16 ||
        t.ic < 1 || t.ic > 15 || 2 * (size_t)t.ic * (t.gc + O) * 128 > 227 * 1024)
      return fail(c, EPHDC_EINVAL, "invalid MAC tiling %lld", (long long)v);
    c->tile = t;
  } else {
    return fail(c, EPHDC_EINVAL, "unknown knob %s", knob);
  }
  return EPHDC_OK;
}

int64_t ephdc_tune_get(const ephdc_ctx* c, const char* knob) {
  if (!c || !knob) return -1;
  if (!strcmp(knob, "mac_mode")) return c->mac_mode;
  if (!strcmp(knob, "mac_min_groups")) return c->mac_min_groups;
  if (!strcmp(knob, "mac_tc_min_groups")) return c->mac_tc_min_groups;
  if (!strcmp(knob, "ntt_plan")) return c->dc.ntt_plan;
  if (!strcmp(knob, "layout")) return c->dc.layout;
  if (!strcmp(knob, "model_digits")) return c->dc.mdig;
  if (!strcmp(knob, "mac_cluster")) return c->mac_cluster;
  if (!strcmp(knob, "chunk")) return c->chunk;
  if (!strcmp(knob, "model_seed")) return c->dc.compact ? (int64_t)c->dc.model_seed : -1;
  if (!strcmp(knob, "hdc_mode")) return c->dc.hdc_mode;
  if (!strcmp(knob, "mac_splits")) return c->mac_splits;
  if (!strcmp(knob, "mac_tile"))
    return (int64_t)c->tile.gt * 1000000 + c->tile.ot * 10000 + c->tile.gc * 100 + c->tile.ic;
  return -1;
}

ephdc_status ephdc_device_status(ephdc_ctx* c) {
  CHECK_CTX(c);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(c, e, "device_status");
  uint32_t word = 0;
  e = cudaMemcpy(&word, c->dc.status, sizeof word, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(c, e, "device_status");
  if (word) {
    cudaMemset(c->dc.status, 0, sizeof word);
    return fail(c, EPHDC_ETIMEOUT, "a bounded device wait gave up (code %u)", word);
  }
  return EPHDC_OK;
}

ephdc_status ephdc_wait_selfcheck(ephdc_ctx* c, int64_t limit_cycles, void* stream) {
  CHECK_CTX(c);
  if (limit_cycles < 1 || limit_cycles > (1ll << 31))
    return fail(c, EPHDC_EINVAL, "limit_cycles must be in [1, 2^31]");
  return launched(c, ephdc::launch_wait_selfcheck(c->dc, (long long)limit_cycles,
                                                  EPHDC_SELFCHECK_WAIT_CODE,
                                                  (cudaStream_t)stream),
                  "wait_selfcheck");
}

ephdc_status ephdc_profile_enable(ephdc_ctx* c, int on) {
  CHECK_CTX(c);
  c->prof = on != 0;
  return EPHDC_OK;
}

ephdc_status ephdc_profile_read(ephdc_ctx* c, double* ms, uint64_t* calls, uint64_t* launches) {
  CHECK_CTX(c);
  if (!ms) return fail(c, EPHDC_EINVAL, "ms is NULL");
  for (int i = 0; i < EPHDC_NSTAGES; i++) {
    ms[i] = 0.0;
    if (calls) calls[i] = 0;
  }
  cudaError_t err = cudaSuccess;
  for (auto& r : c->recs) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    ms[r.stage] += t;
    if (calls) calls[r.stage]++;
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->recs.clear();
  if (launches) *launches = c->launches;
  c->launches = 0;
  return cuda_status(c, err, "profile_read");
}

}  // extern "C"

namespace ephdc {
const DevCtx* ctx_dev(const ephdc_ctx* c) { return &c->dc; }
int ctx_device(const ephdc_ctx* c) { return c->device; }
ephdc_status ctx_fail(ephdc_ctx* c, ephdc_status s, const char* msg) { return fail(c, s, "%s", msg); }
void ctx_clear_error(ephdc_ctx* c) { c->err.clear(); }
}  // namespace ephdc
