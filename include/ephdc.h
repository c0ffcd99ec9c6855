/*
 * ephdc.h -- C ABI of the GB300 (sm_103a) EP-HDC client-side inference library.
 *
 * EP-HDC ("Hyperdimensional Computing with Encrypted Parameters") runs HDC
 * inference on the client against a BFV-encrypted model (Sec. 4.1): the client
 * encodes its samples into quantised hypervectors in plaintext (Sec. 2.1,
 * Sec. 5.1), batch-encodes element d of many query hypervectors into the SIMD
 * slots of one plaintext (Sec. 3, the SIMD representation), multiplies the
 * plaintexts with the encrypted class hypervectors and accumulates (Sec. 4.1,
 * "HE compute"), and returns one ciphertext of similarity scores per batch.
 * Galois rotation with key switching (Sec. 2.2) folds D-chunks that share a
 * plaintext into the per-class score.
 *
 * Conventions for every entry point:
 *  - All pointers named *_dev are device pointers owned by the caller; sizes come
 *    from the ephdc_*_bytes queries.  Device pointers must be 16-byte aligned.
 *    The library owns only its context (tables, scratch workspace).
 *  - Work is enqueued asynchronously on the given CUDA stream (NULL = legacy
 *    default stream).  Argument errors are detected on the host before anything is
 *    enqueued and return EPHDC_EINVAL (or EPHDC_EUNSUPPORTED) with a message in
 *    ephdc_last_error(); launch failures return EPHDC_ECUDA.
 *  - A context is not thread-safe: use one context per host thread (or serialise).
 *  - No exception crosses the ABI.  No call falls back to the CPU.
 *  - Ciphertexts exchanged with the host ("coefficient domain") are u32 words in
 *    [0, q_l), layout [2 polys][L limbs][n coefficients]; the number-theoretic-
 *    transform (NTT) domain storage order of device buffers is private.
 *
 * Parameters: ring degree n (power of two, 1024..16384), L RNS primes q_l < 2^30
 * with q_l = 1 (mod 2n) (the L largest such primes), plaintext modulus t = 65537,
 * ternary secret, discrete Gaussian error (sigma, support [-19, 19]).
 * Slot layout (k_in, r): each plaintext carries r consecutive elements of every
 * query hypervector (D-chunks); a chunk spans W = n/(2r) slots of each of the two
 * slot rows and holds k_in classes side by side, cap_row = floor(W / k_in) queries
 * each; a group of cap = 2*cap_row queries needs P = ceil(D/r) plaintexts.
 * r = 1 with k_in = k is the paper's representation (batch floor(N/k), D MulCP,
 * no rotation); r > 1 adds log2(r) rotations per output ciphertext.
 */
#ifndef EPHDC_H
#define EPHDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EPHDC_OK = 0,
  EPHDC_EINVAL = -1,       /* bad argument (size, pointer, alignment, parameter)   */
  EPHDC_EUNSUPPORTED = -2, /* valid but not supported by this library             */
  EPHDC_ENOMEM = -3,       /* device allocation failed / batch above the reserve  */
  EPHDC_ECUDA = -4,        /* a CUDA call or kernel launch failed                 */
  EPHDC_ETIMEOUT = -5,     /* a bounded device wait gave up                       */
  EPHDC_EBUSY = -6         /* resource in use                                      */
} ephdc_status;

typedef struct {
  uint32_t n;         /* ring degree, power of two in [1024, 16384]               */
  uint32_t L;         /* number of RNS primes, 2..8                               */
  uint32_t k;         /* number of classes                                        */
  uint32_t k_in;      /* classes packed per ciphertext (divides k)                */
  uint32_t r;         /* D-chunks folded per plaintext (power of two)            */
  uint32_t D;         /* hypervector dimension                                     */
  uint32_t F;         /* feature count (multiple of 16)                           */
  uint32_t hv_bits;   /* query hypervector precision b, 2..8                      */
  int32_t shift;      /* quantiser shift s >= 0                                   */
  uint32_t max_batch; /* largest batch B any call on this context will use        */
  double sigma;       /* error standard deviation (3.2)                           */
  uint32_t t;         /* plaintext modulus: a prime = 1 (mod 2n) below the smallest
                         RNS prime; 0 selects 65537                                */
  uint32_t prime_bits;/* the L RNS primes are the largest primes below 2^prime_bits
                         with q = 1 (mod 2n); 20..30, 0 selects 30                 */
  uint32_t scale_shift; /* scaling operation of Sec. 5.1: 0 = off; else the running
                         accumulator is multiplied by (2^scale_shift)^-1 mod t
                         after every scale_group additions                         */
  uint32_t scale_group; /* g of the scaling operation (0 selects 512)              */
} ephdc_params;

typedef struct ephdc_ctx ephdc_ctx; /* opaque, owned by the library */

/* Create a context: validates params, derives primes, roots, twiddle and slot
 * tables, and reserves scratch for batches up to params->max_batch.  Returns
 * EPHDC_EINVAL for invalid parameters, EPHDC_ENOMEM if device memory runs out,
 * EPHDC_ECUDA if no device is usable.  *out is NULL on failure. */
ephdc_status ephdc_ctx_create(const ephdc_params* params, ephdc_ctx** out);
void ephdc_ctx_destroy(ephdc_ctx* ctx);
/* Message of the last failing call on this context ("" if none); valid until the
 * next call on the context.  ctx may be NULL (message of the last failed create). */
const char* ephdc_last_error(const ephdc_ctx* ctx);

/* Derived quantities: which = "cap" (queries per group), "P" (plaintexts per
 * group), "Kp" (ciphertexts per plaintext index = k/k_in), "W", "cap_row",
 * "logr", "t" (the plaintext modulus), "q0".."q7" (the primes).  Returns 0 for an
 * unknown name. */
uint64_t ephdc_query(const ephdc_ctx* ctx, const char* which);

/* Buffer sizes in bytes. */
size_t ephdc_sk_bytes(const ephdc_ctx* ctx);          /* secret key (server)          */
size_t ephdc_galois_key_bytes(const ephdc_ctx* ctx);  /* log2(r) rotation keys         */
size_t ephdc_model_bytes(const ephdc_ctx* ctx);       /* encrypted class hypervectors */
size_t ephdc_plain_bytes(const ephdc_ctx* ctx, int32_t B);   /* bfv_encode_plain out  */
size_t ephdc_out_ct_bytes(const ephdc_ctx* ctx, int32_t B);  /* score ciphertexts     */

/* ---------------------------------------------------------------- server side */
/* Secret key and Galois (rotation) keys from a 64-bit seed.  Sec. 2.2: RLWE secret
 * (ternary) and key-switching keys for the rotations of rotate-and-sum, one per
 * fold step j < log2 r (Galois element 3^(W*2^j) mod 2n), BV decomposition over the
 * L RNS digits.  Randomness: ChaCha20 (RFC 8439) keyed by the seed.
 * sk_dev: ephdc_sk_bytes; gk_dev: ephdc_galois_key_bytes (may be NULL if r = 1). */
ephdc_status bfv_keygen(ephdc_ctx* ctx, uint64_t seed, void* sk_dev, void* gk_dev,
                        void* stream);

/* Encrypt the k class hypervectors (Sec. 4.1: the model, not the queries, is
 * encrypted).  class_hv_dev: int8 [k][D] row-major.  Secret-key BFV encryption:
 * c1 = a, c0 = -a*s + e + round(q*m/t) per ciphertext (m in [0, t), ties rounded up),
 * slots laid out per (k_in, r).
 * model_dev: ephdc_model_bytes, device-private NTT-domain order. */
ephdc_status bfv_encrypt_model(ephdc_ctx* ctx, const int8_t* class_hv_dev, const void* sk_dev,
                               uint64_t seed, void* model_dev, void* stream);

/* Decrypt score ciphertexts (checking only; needs the server's secret key).
 * out_ct_dev: as written by bfv_ptct_similarity / ephdc_infer for a batch of B.
 * scores_dev: uint32 [B][k], values in [0, t): sum_d h[d] * c_j[d] mod t. */
ephdc_status bfv_decrypt_scores(ephdc_ctx* ctx, const void* sk_dev, const uint32_t* out_ct_dev,
                                int32_t B, uint32_t* scores_dev, void* stream);

/* ---------------------------------------------------------------- client hot path */
/* HDC encoding (Sec. 2.1 random projection) with quantisation (Sec. 5.1):
 * A = X * Wt^T exactly in int32, H = clamp(floor((A + 2^(s-1)) / 2^s), -2^(b-1),
 * 2^(b-1)-1).  X_dev: int8 [B][F]; Wt_dev: int8 [D][F] (row d = weights of
 * dimension d); H_dev: int8 [B][D].  1 <= B <= max_batch.  The product runs on the
 * tensor cores in fp16 x fp16 -> fp32, which is exact here: operands are integers of
 * magnitude <= 128 and every partial sum stays below 2^24 (F <= 65536). */
ephdc_status hdc_encode(ephdc_ctx* ctx, const int8_t* X_dev, const int8_t* Wt_dev, int32_t B,
                        int8_t* H_dev, void* stream);

/* Batch-encode query hypervectors into BFV plaintexts (EncPt): slot packing per
 * (k_in, r), inverse NTT mod t (slot -> coefficient), centred lift and forward
 * NTT per RNS limb.  H_dev: int8 [B][D] (with r = 8 or 16 at k_in = 1, or r = 4 at
 * k_in = 2, and D a multiple of r, query rows are read by vector loads; other layouts
 * byte by byte, same result).  pt_dev: ephdc_plain_bytes(B). */
ephdc_status bfv_encode_plain(ephdc_ctx* ctx, const int8_t* H_dev, int32_t B, uint32_t* pt_dev,
                              void* stream);

/* Encrypted similarity (HE compute, Sec. 4.1): for every group g and ciphertext
 * column j', acc = sum_i pt[g][i] * model[i][j'] (pt x ct multiply-accumulate over
 * the RNS limbs), then log2(r) rotate-and-sum steps with key switching, then the
 * inverse NTT to the coefficient domain.  out_ct_dev: uint32 [G][k/k_in][2][L][n],
 * G = ceil(B / cap).  gk_dev may be NULL if r = 1. */
ephdc_status bfv_ptct_similarity(ephdc_ctx* ctx, const uint32_t* pt_dev, int32_t B,
                                 const void* model_dev, const void* gk_dev, uint32_t* out_ct_dev,
                                 void* stream);

/* Same result as bfv_ptct_similarity, bit for bit, for callers that must not
 * allocate device memory while they serve: a serving loop whose admission control
 * has already budgeted every byte of HBM, a process whose memory pool owns the
 * device, or a latency-critical loop that cannot afford the device-wide
 * synchronisation a cudaMalloc/cudaFree can cause.  The paper has no counterpart;
 * it is an interface of this library only.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.  Its
 *    scratch is one array of EPHDC_STATIC_SCRATCH_BYTES (8 MiB) compiled into the
 *    library as a __device__ variable, which every GPU that loads the library holds
 *    until the process exits.  The context must still be created beforehand (that
 *    call allocates the context's tables).
 *  - Every call looks up the array's device address on the current device (a host
 *    query, so it stays valid when a cudaDeviceReset loads the module anew); the
 *    first call on a device may load the module, so make it before any stream
 *    capture.
 *  - All calls share the one array, and it keeps the last call's contents (nothing
 *    in it needs to start at zero).  Calls whose work overlaps on the GPU -- on
 *    different streams, or from different contexts on the same device -- race on
 *    it: serialise them.
 *  - A batch is rejected with EPHDC_EINVAL before anything is enqueued when its
 *    scratch exceeds the array.  With C = G * (k/k_in) score ciphertexts of 2*L*n
 *    words each (G = ceil(B / cap)), the scratch is two accumulator sets (2 C
 *    ciphertexts), the key-switch digits (C * L * n words, half a set) and at least
 *    one split of partial sums (C ciphertexts): 28 * C * L * n bytes.  With n = 8192
 *    and L = 4 that allows C <= 9.
 * Arguments as for bfv_ptct_similarity. */
#define EPHDC_STATIC_SCRATCH_BYTES (8u << 20)
ephdc_status bfv_ptct_similarity_noalloc(ephdc_ctx* ctx, const uint32_t* pt_dev, int32_t B,
                                         const void* model_dev, const void* gk_dev,
                                         uint32_t* out_ct_dev, void* stream);

/* The whole client path in one call: hdc_encode, bfv_encode_plain and
 * bfv_ptct_similarity on context scratch. */
ephdc_status ephdc_infer(ephdc_ctx* ctx, const int8_t* X_dev, const int8_t* Wt_dev, int32_t B,
                         const void* model_dev, const void* gk_dev, uint32_t* out_ct_dev,
                         void* stream);

/* ---------------------------------------------------------------- batching */
/* One client's queries: B rows of F int8 features at X_dev (B may be 0). */
typedef struct {
  const int8_t* X_dev;
  int32_t B;
} ephdc_request;

/* Many clients' uneven batches in one pass (Sec. 3: batch inference fills the SIMD
 * slots).  The requests are packed back to back into one query space of
 * B = sum B_r <= max_batch queries: request r owns queries [off_r, off_r + B_r),
 * off_r = sum_{r' < r} B_r', so its scores sit in groups off_r / cap ...; one pass
 * reads the encrypted model once for all groups.  out_ct_dev: as ephdc_infer for B
 * queries.  Each request's decrypted scores equal those of running it alone. */
ephdc_status ephdc_infer_multi(ephdc_ctx* ctx, const ephdc_request* reqs, int32_t nreq,
                               const int8_t* Wt_dev, const void* model_dev, const void* gk_dev,
                               uint32_t* out_ct_dev, void* stream);

/* ---------------------------------------------------------------- seeded model message */
/* The encrypted model is sent once, server to client (Sec. 4.1).  Every model
 * ciphertext's c1 is the uniform polynomial a drawn from ChaCha20 (domain 2,
 * ciphertext number i*Kp + jp, keyed by the encryption seed), so the message can be
 * c0 alone plus the 8-byte seed: half the bytes of the full model.  The client
 * rebuilds the identical device model once, at load time.
 * seeded_dev: ephdc_model_seeded_bytes(), [P*Kp][L][n] u32, coefficient domain. */
size_t ephdc_model_seeded_bytes(const ephdc_ctx* ctx);
/* Server: the c0 halves of model_dev (from bfv_encrypt_model) as the seeded message. */
ephdc_status bfv_model_to_seeded(ephdc_ctx* ctx, const void* model_dev, uint32_t* seeded_dev,
                                 void* stream);
/* Client: model_dev (ephdc_model_bytes) from the seeded message and the seed it was
 * encrypted with; equal word for word to the model bfv_encrypt_model produced. */
ephdc_status bfv_model_from_seeded(ephdc_ctx* ctx, const uint32_t* seeded_dev, uint64_t seed,
                                   void* model_dev, void* stream);

/* Client: the digit model (see the knob "model_digits") from a model in the standard
 * device order, model_dev as bfv_encrypt_model produces it with "model_digits" 0 and
 * "layout" 0 ([P][k/k_in][2][L][n] NTT-domain residues, ephdc_model_bytes of such a
 * context); model_digits_dev holds ephdc_model_bytes of this context, which must have
 * "model_digits" 1 (else EPHDC_EUNSUPPORTED).  Equal to what bfv_encrypt_model writes
 * for the same ciphertexts under "model_digits" 1. */
ephdc_status bfv_model_to_digits(ephdc_ctx* ctx, const void* model_dev, void* model_digits_dev,
                                 void* stream);

/* ---------------------------------------------------------------- server-side variant */
/* HE-HDC-SR (Sec. 3, the comparison of Sec. 6, Table t:clientrt): the roles of the
 * client-side path swapped.  The CLIENT holds the secret key and encrypts its query
 * hypervectors in the SIMD form (one ciphertext per query plaintext, G*P of them per
 * batch); the SERVER holds the class hypervectors as plaintexts, computes the same
 * dot products ct x pt, rotates-and-sums, and returns G*(k/k_in) score ciphertexts
 * that the client decrypts with bfv_decrypt_scores.  Same parameters, slot layout,
 * Galois keys and output format as the client-side path. */
size_t ephdc_query_ct_bytes(const ephdc_ctx* ctx, int32_t B); /* G*P ciphertexts        */
size_t ephdc_model_plain_bytes(const ephdc_ctx* ctx);         /* (k/k_in)*P plaintexts  */

/* Client: secret-key encryption of query plaintext (g, i) (its slots as in
 * bfv_encode_plain): c1 = a, c0 = -a s + e + round(q m / t).  Randomness: ChaCha20
 * keyed by the seed, ciphertext number g*P + i, domain 6 (a) and 7 (e).
 * H_dev: int8 [B][D], 1 <= B <= max_batch.  query_ct_dev: ephdc_query_ct_bytes(B),
 * [G][P][2][L][n] in the device NTT order (ephdc_ct_to_host_coeff reads it).
 * Caller-owned, 16-byte aligned; EPHDC_EINVAL / EPHDC_ENOMEM as bfv_encode_plain. */
ephdc_status bfv_encrypt_queries(ephdc_ctx* ctx, const int8_t* H_dev, int32_t B,
                                 const void* sk_dev, uint64_t seed, uint32_t* query_ct_dev,
                                 void* stream);
/* Server (setup): class hypervector (jp*k_in + jin) as plaintexts mm[jp][i] holding
 * c[i*r + ch] in slot (rho, ch*W + jin*cap_row + qq) for every qq < cap_row.
 * class_hv_dev: int8 [k][D].  model_plain_dev: ephdc_model_plain_bytes(),
 * [k/k_in][P][L][n] in the device NTT order (ephdc_plain_to_host_coeff reads it). */
ephdc_status bfv_encode_model_plain(ephdc_ctx* ctx, const int8_t* class_hv_dev,
                                    uint32_t* model_plain_dev, void* stream);
/* Server: Acc[g][jp] = sum_i query_ct[g][i] * mm[jp][i] (negacyclic, per limb), then
 * the rotate-and-sum and the export of ephdc_infer.  out_ct_dev:
 * ephdc_out_ct_bytes(B), coefficient domain.  Uses the context's scratch. */
ephdc_status bfv_ctpt_similarity(ephdc_ctx* ctx, const uint32_t* query_ct_dev, int32_t B,
                                 const uint32_t* model_plain_dev, const void* gk_dev,
                                 uint32_t* out_ct_dev, void* stream);

/* ---------------------------------------------------------------- noise growth */
/* One trial of the noise-growth experiment (Sec. 5.2, Alg. 1 findDmax): how many
 * plaintext x ciphertext products the accumulator takes before decryption fails.
 * Needs the paper's layout with one class (k = k_in = 1, r = 1) and one group of
 * 1 <= B <= cap queries; pt_dev = bfv_encode_plain(H_dev) and model_dev =
 * bfv_encrypt_model(class_hv_dev) for the context's D dimensions, sk_dev their key.
 * The accumulator after D' products (D' = 1..D) is the evaluation with D'
 * dimensions; each is decrypted and compared with sum_{d < D'} h[q][d] c[d] mod t
 * for every query q.  *dmax = the largest D' such that every evaluation with
 * 1..D' dimensions is correct (D if none fails).  Synchronous on the default
 * stream; allocates and frees D (L n + n) words of device scratch.  EPHDC_EUNSUPPORTED
 * for another layout, EPHDC_EINVAL for a bad B or pointer. */
ephdc_status ephdc_find_dmax_trial(ephdc_ctx* ctx, const void* sk_dev, const int8_t* H_dev,
                                   int32_t B, const int8_t* class_hv_dev, const uint32_t* pt_dev,
                                   const void* model_dev, int32_t* dmax);

/* Schedule knobs of the multi-accumulate (set by the autotuner; results never
 * change): "mac_mode" 0 automatic / 1 streaming / 2 tiled / 3 tensor cores (exact
 * signed-digit split, k/k_in <= 16) / 4 tensor cores on the digit model (see
 * "model_digits"), "mac_cluster" 0, 1, 2, 4 or 8 (the digit-model product: CTAs of
 * consecutive group blocks that share each model block by multicast, 0 = 4), "mac_min_groups" and "mac_tc_min_groups" (tiled, tensor
 * cores from this many groups on in automatic mode), "mac_splits" (streaming split cap, 0 =
 * heuristic), "mac_tile" = gt*10^6 + ot*10^4 + gc*100 + ic (groups and outputs per
 * warp, groups per CTA, plaintexts per staged chunk, at most 15); "hdc_mode" 0..4 is
 * the HDC projection kernel (persistent tensor-core GEMM with 128 x 256 tiles and a
 * 3-stage ring / one 128 x 128 tile per CTA / persistent with 128 x 128 tiles /
 * persistent 128 x 256 with a 4-stage ring / mode 0 in clusters of two CTAs that take
 * row blocks 2m and 2m + 1 of the same 256 columns and share each W slice by multicast);
 * "ntt_plan" 0/1/2
 * is the pass schedule of the encoding transforms (balanced, radix-32 passes first,
 * radix-32 passes last).  "layout" 0/1 is the device order of the NTT-domain
 * plaintexts and model: 0 = [G][P][L][n] and [P][k/k_in][2][L][n]; 1 = blocked by 4
 * coefficients, [L][n/4][G][P][4] and [L][n/4][P][2 k/k_in][4] (needs k/k_in <= 16),
 * read by the tensor-core product with every tile's data contiguous.  Set "layout"
 * before bfv_encrypt_model: a model is only valid for contexts with the layout it was
 * encrypted under.  With layout 1 the multiply-accumulate always runs on the tensor
 * cores ("mac_mode" 1 or 2 fails with EPHDC_EUNSUPPORTED), and the seeded model message,
 * the server-side variant, the noise-growth trial and bfv_ptct_similarity_noalloc
 * return EPHDC_EUNSUPPORTED.  "chunk" c > 0 makes ephdc_infer, when it runs the tiled
 * multi-accumulate with layout 0 and no scaling operation, encode and accumulate
 * plaintext indices [i0, i0 + c) of every group at a time in the plaintext scratch
 * instead of the whole pass (same results; measured slower on GB300); 0 = off.
 * "model_seed" s >= 0 selects the compact model (Sec. 4.1: the model is shipped once;
 * here only c0 is ever stored, ephdc_model_bytes halves): bfv_encrypt_model draws c1 in
 * the evaluation domain, device position k of limb l = word64(l n + k) mod q_l of the
 * ChaCha20 stream (s, domain 8, ciphertext number), and stores c0 only, [P][k/k_in][L][n];
 * the tiled multiply-accumulate regenerates c1 from s as it stages the model (the
 * automatic and the tiled "mac_mode" only).  -1 (the default) = the full model.  Set it,
 * with the seed the model is encrypted with, on every context that uses the model and
 * before bfv_encrypt_model; the blocked layout, the seeded model message, the noise-growth
 * trial and bfv_ptct_similarity_noalloc do not take it (EPHDC_EUNSUPPORTED).
 * "model_digits" 1 selects the digit model (needs k/k_in <= 16, layout 0 and the full
 * model): the model is stored as the fp16 tensor-core operand of the signed base-256
 * digits d_v of every residue (x = sum_{v<4} d_v 2^(8v), d_v = byte v of x + 0x80808080
 * less 128, |d_v| <= 128), so that the multiply-accumulate copies it into shared memory
 * without splitting it; ephdc_model_bytes = L n ceil(P/16) 32 R with R = 64 rows when
 * k/k_in <= 8, else 128 (twice the residue model at k/k_in = 16 or 8).  Order: fp16
 * tiles of R rows x 16 columns, tile ((l (n/8) + x/8) ceil(P/16) + i/16) 8 + x%8 for
 * coefficient x of limb l and plaintext i; row 4 o + v, column i%16 at byte
 * (row/8) 256 + (column/8) 128 + (row%8) 16 + (column%8) 2; rows of outputs
 * o >= 2 k/k_in and columns of plaintexts i >= P are zero.
 * Set it before bfv_encrypt_model (or convert a residue model with
 * bfv_model_to_digits); the multiply-accumulate then runs "mac_mode" 4 (0 or 4 accepted,
 * others EPHDC_EUNSUPPORTED), and the seeded model message, the compact model, the
 * blocked layout, the noise-growth trial and bfv_ptct_similarity_noalloc return
 * EPHDC_EUNSUPPORTED.  ephdc_model_to_host_coeff reassembles the residues.
 * EPHDC_EINVAL for an unknown knob or an invalid value.  ephdc_tune_get returns -1 for
 * an unknown knob. */
ephdc_status ephdc_tune_set(ephdc_ctx* ctx, const char* knob, int64_t value);
int64_t ephdc_tune_get(const ephdc_ctx* ctx, const char* knob);

/* ---------------------------------------------------------------- host formats */
/* Copy `count` device NTT-domain ciphertexts (e.g. the model, [2][L][n] each) to
 * the host in the coefficient domain, uint32 [count][2][L][n].  Synchronous. */
ephdc_status ephdc_ct_to_host_coeff(ephdc_ctx* ctx, const void* ct_dev, int32_t count,
                                    uint32_t* host);
/* The secret key as n signed coefficients in {-1, 0, 1} on the host.  Synchronous. */
ephdc_status ephdc_sk_to_host(ephdc_ctx* ctx, const void* sk_dev, int32_t* host);
/* Galois keys to the host, uint32 [log2 r][L digits][2][L limbs][n] coefficient
 * domain.  Synchronous. */
ephdc_status ephdc_gk_to_host_coeff(ephdc_ctx* ctx, const void* gk_dev, uint32_t* host);
/* The encrypted model (either layout) to the host in the coefficient domain, uint32
 * [P][k/k_in][2][L][n].  Synchronous; allocates temporary device memory. */
ephdc_status ephdc_model_to_host_coeff(ephdc_ctx* ctx, const void* model_dev, uint32_t* host);
/* Plaintexts from bfv_encode_plain to the host as the lifted plaintext polynomial
 * per limb, uint32 [count][L][n] in [0, q_l); with layout 1, count must be a whole
 * number of groups (G * P).  Synchronous. */
ephdc_status ephdc_plain_to_host_coeff(ephdc_ctx* ctx, const uint32_t* pt_dev, int32_t count,
                                       uint32_t* host);

/* Forward (inverse = 0) or inverse (inverse = 1) negacyclic NTT of `count`
 * polynomials mod q_limb (limb = L selects t), in place on the device, with the
 * evaluation vector in natural order: a_hat[j] = a(psi^(2j+1)).  For checking the
 * transform against other implementations. */
ephdc_status ephdc_ntt_natural(ephdc_ctx* ctx, uint32_t limb, uint32_t* poly_dev, int32_t count,
                               int inverse, void* stream);

/* Pipeline waits inside the kernels (tensor-core producer/consumer barriers) are
 * bounded: a wait that gives up records a code in the context's device status word,
 * the kernel skips its remaining work and returns, and the context stays usable.
 * This call waits for all work on the device and returns EPHDC_ETIMEOUT (clearing
 * the word) if any wait gave up since the last call, else EPHDC_OK. */
ephdc_status ephdc_device_status(ephdc_ctx* ctx);

/* Self-check of the bounded waits above (failure detection): enqueues on `stream`
 * one single-thread kernel that initialises an mbarrier nothing ever arrives on and
 * waits for it through the same bounded-wait routine as the tensor-core pipelines,
 * giving up after limit_cycles SM clock cycles (1 .. 2^31; 10^5 is about 50 us).
 * No copy or MMA is in flight while it waits.  The next ephdc_device_status then
 * returns EPHDC_ETIMEOUT with code EPHDC_SELFCHECK_WAIT_CODE in its message, and the
 * context stays usable.  The paper has no counterpart.  EPHDC_EINVAL for a limit
 * out of range. */
#define EPHDC_SELFCHECK_WAIT_CODE 99u
ephdc_status ephdc_wait_selfcheck(ephdc_ctx* ctx, int64_t limit_cycles, void* stream);

/* ---------------------------------------------------------------- measurement */
/* Stages of the client path, for per-stage device timing. */
enum {
  EPHDC_STAGE_HDC = 0,     /* hdc_encode                                   */
  EPHDC_STAGE_ENCODE = 1,  /* bfv_encode_plain                             */
  EPHDC_STAGE_MAC = 2,     /* pt x ct multiply-accumulate (+ split reduce) */
  EPHDC_STAGE_ROTATE = 3,  /* rotate-and-sum with key switching            */
  EPHDC_STAGE_EXPORT = 4,  /* inverse NTT of the score ciphertexts         */
  EPHDC_STAGE_ENCRYPT = 5, /* bfv_encrypt_queries (server-side variant)    */
  EPHDC_NSTAGES = 6
};
/* When on, every client-path call records a CUDA event pair around each stage on the
 * call's own stream (no synchronisation).  Off by default. */
ephdc_status ephdc_profile_enable(ephdc_ctx* ctx, int on);
/* Waits for the recorded events, writes the summed device milliseconds per stage
 * (ms[EPHDC_NSTAGES]), the number of recorded calls per stage (calls[EPHDC_NSTAGES],
 * may be NULL) and the number of kernel launches the library has enqueued since the
 * last read (*launches, may be NULL), then clears the record. */
ephdc_status ephdc_profile_read(ephdc_ctx* ctx, double* ms, uint64_t* calls, uint64_t* launches);

/* Integer-pipe peaks of the current device, measured by two register-only kernels:
 * *bfly_per_s = lazy Harvey forward butterflies with a Shoup quotient per second
 * (the transforms' instruction mix), *mac_per_s = 64-bit carry-chain
 * multiply-accumulates (mad.lo.cc + madc.hi) per second.  Synchronous, about 30 ms
 * of device time; allocates and frees a small buffer.  Not part of the method: the
 * denominators of the integer-bound rooflines.  EPHDC_EINVAL for NULL outputs,
 * EPHDC_ENOMEM / EPHDC_ECUDA on device errors. */
ephdc_status ephdc_measure_int_peaks(double* bfly_per_s, double* mac_per_s);

#ifdef __cplusplus
}
#endif
#endif /* EPHDC_H */
