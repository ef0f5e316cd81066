/*
 * fhe.h -- C ABI of libfhe: RNS-CKKS evaluation of neural-network graphs on one
 * NVIDIA GB300 (sm_103a), after arXiv 2110.13638 ("EDLaaS: Fully Homomorphic
 * Encryption Over Neural Network Graphs").
 *
 * Conventions (every entry point):
 *   - returns int: FHE_OK (0) or a negative FHE_E* code; fhe_last_error()
 *     then holds a message for the calling thread;
 *   - handles (fhe_ctx, fhe_graph) are opaque, owned by the library and freed
 *     by their *_destroy call;
 *   - pointers named d_* are DEVICE pointers owned by the caller (e.g. the
 *     storage of a PyTorch tensor); the library never frees them.  Pointers
 *     named h_* or plain arrays are HOST memory owned by the caller and read
 *     only during the call;
 *   - `stream` is a cudaStream_t (NULL = legacy default stream); device work is
 *     enqueued on it and the call returns without waiting unless stated;
 *   - one context must not be used from two streams or threads at once (its
 *     workspace is shared by the calls made on it); forks of one parameter
 *     set (fhe_ctx_fork) may run concurrently.  Keys (fhe_keygen,
 *     fhe_galois_keygen) are generated on the parent before its forks use
 *     them; the packed convolution generates its missing rotation keys on
 *     first use, so run one batch of a graph that has it before forking;
 *   - growing a workspace or batch area (the first call at a larger size)
 *     synchronises the device before freeing the old buffer; size them with
 *     one call before stream capture or latency-critical use;
 *   - every wait a kernel makes on the device is bounded.  A kernel whose wait
 *     gives up leaves its outputs unwritten and sets the context's status
 *     word; FHE_ETIMEOUT then comes from the first of fhe_eval_graph,
 *     fhe_eval_batch or fhe_ctx_sync on that context to run after that kernel
 *     has finished (fhe_ctx_sync waits for the stream, so it always sees it).
 *
 * Data layout:
 *   residue polynomial  : N u64 words, every word < its prime
 *   ciphertext batch    : u64 [n_ct][2][L][N], NTT form (bit-reversed order),
 *                         residue r belongs to prime q_r; L = level
 *   plaintext batch     : u64 [n_ct][L][N], NTT form
 *   coefficient export  : same shapes in coefficient (natural) order
 *   slots               : double [n_ct][N/2] (real slots, batch-in-slots)
 *   decrypted poly      : int64 [n_ct][N], centred coefficients mod q_0
 */
#ifndef FHE_H
#define FHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FHE_OK 0
#define FHE_EINVAL (-1)       /* bad argument, shape or graph */
#define FHE_ENOMEM (-2)       /* device or host allocation failed */
#define FHE_ELEVEL (-3)       /* not enough primes left for the operation */
#define FHE_ESCALE (-4)       /* operands' nominal scales disagree */
#define FHE_ECUDA (-5)        /* a CUDA runtime call failed */
#define FHE_ETIMEOUT (-6)     /* a bounded device wait gave up */
#define FHE_EUNSUPPORTED (-7) /* valid request this build does not implement */
#define FHE_ENOKEY (-8)       /* fhe_keygen has not run on this context */

typedef struct fhe_ctx fhe_ctx;
typedef struct fhe_graph fhe_graph;

/* Context facts (fhe_ctx_query). */
typedef struct {
    uint32_t N;          /* ring degree */
    uint32_t slots;      /* N / 2 */
    uint32_t L_top;      /* data primes q_0 .. q_{L_top-1} */
    uint32_t log_scale;  /* scale = 2^log_scale */
    uint64_t primes[64]; /* q_0 .. q_{L_top-1}, then the special prime P */
    uint64_t key_bytes;  /* device bytes held for keys and tables */
    uint32_t ntt_variant;        /* NTT schedule the autotuner picked (0..5) */
    float ntt_variant_us[16];    /* autotuner: microseconds per transform of each schedule (0 = not timed) */
    uint32_t ntt_variant_ks;     /* schedule of the key-switching inner-product transforms (0..7) */
    float ntt_variant_ks_us[16]; /* autotuner: microseconds per digit transform of each schedule */
    uint64_t workspace_bytes;    /* device bytes of this context's call workspace and batch
                                    area (both grow on demand; 0 before the first call that
                                    needs them) */
} fhe_ctx_info;

/* Per-ciphertext metadata returned by graph evaluation. */
typedef struct {
    uint32_t level;      /* number of primes held */
    double scale;        /* nominal scale (FP64) */
} fhe_ct_meta;

/* ---- graph description (host arrays, copied by fhe_graph_create) ---------
 * Sec. 3 graph rules: nodes are blocks (layers); an edge carries a list of
 * ciphertexts; a node with several in-edges sees them stacked in edge order
 * (FHE_NODE_ADD sums them element by element instead); a node fires once all
 * in-edges carry data; its output goes to every out-edge. */
enum {
    FHE_NODE_INPUT = 0,  /* source: encrypted input signal (type of concern) */
    FHE_NODE_LINEAR = 1, /* y_o = sum_e w_e x_{col_e} + b_o (dense or conv), cost 1 */
    FHE_NODE_POLY = 2,   /* sum_i a_i x^i per ciphertext, degree 1..31: degree 1 cost 1,
                            2 and 3 cost 2 (dedicated schedules), 4..31 cost
                            ceil(log2 degree) + 1 (powers by products, one combining
                            rescale) */
    FHE_NODE_SQUARE = 3, /* x^2 per ciphertext, cost 1 */
    FHE_NODE_ADD = 4,    /* element-wise sum of the in-edge lists, cost 0 */
    FHE_NODE_OUTPUT = 5, /* sink: result handed to the client (type of concern) */
    FHE_NODE_RELU = 6,   /* Eq. relu_approximate with range q = coeffs[0]:
                            4/(3 pi q) x^2 + x/2 + q/(3 pi), a degree-2 POLY, cost 2 */
    FHE_NODE_ROTATE = 7, /* rotation (client refresh, Sec. 3.1): a concern node where the
                            ciphertexts go back to the client to be decrypted and
                            re-encrypted; it ends one parameter group and starts
                            another.  fhe_eval_graph refuses graphs that contain it:
                            each group is evaluated on its own context. */
    FHE_NODE_CONV_PACKED = 8 /* kernel masquerading (Sec. 3.2) on images packed in slots
                            (image b's pixel (i, j) at slot b S + i W + j): per kernel
                            position the input is rotated by dr W + dc and multiplied
                            slot-wise by the merged mask-and-kernel vector (weight at
                            the valid output slots b S + s r W + s c, zero elsewhere);
                            the k^2 products are summed, rescaled and the bias vector
                            added.  n_out = filters F, weight = [F][k][k], bias = [F],
                            conv = {H, W, k, stride, images per ciphertext, S}; outputs
                            filter-major (F x inputs); needs the rotation keys of the
                            k^2 offsets (generated on first use); cost 1 */
};

typedef struct {
    uint32_t kind;            /* FHE_NODE_* */
    uint32_t n_out;           /* LINEAR: outputs; INPUT: ciphertexts it receives */
    const uint32_t* row_ptr;  /* LINEAR: CSR row pointers, n_out + 1 entries */
    const uint32_t* col_idx;  /* LINEAR: CSR column = index into the stacked input */
    const double* weight;     /* LINEAR: CSR values (FP64) */
    const double* bias;       /* LINEAR: n_out biases (FP64), may be NULL = 0 */
    double coeffs[4];         /* POLY: a0..a_degree; RELU: coeffs[0] = range q > 0 */
    uint32_t degree;          /* POLY: 1..31 (0 means 3) */
    uint32_t conv[6];         /* CONV_PACKED: H, W, k, stride, images, slot stride S */
    const double* coeffs_hi;  /* POLY of degree > 3: a_0 .. a_degree */
} fhe_node_desc;

typedef struct {
    uint32_t n_nodes;
    const fhe_node_desc* nodes;
    uint32_t n_edges;
    const uint32_t* edge_src;   /* edge e goes edge_src[e] -> edge_dst[e] */
    const uint32_t* edge_dst;
} fhe_graph_desc;

/* ---- parameters (Sec. 3.1) ---------------------------------------------- */

/* Alg. parameterise: multiplicative cost c -> ring degree N and the
 * coefficient-modulus bit list m (first and last entries int(s * p); the last
 * one is the special prime).  bits must hold c + 2 entries.  Host only. */
int fhe_parameterise(uint32_t cost, uint32_t log_scale, double special_mult,
                     uint32_t* N, uint32_t* bits, uint32_t bits_cap, uint32_t* n_bits);

/* Alg. autoHE / autoHE_discover over a graph: parameter groups of the
 * ingress nodes (INPUT and ROTATE, the sources of ciphertexts under fresh
 * keys) and each group's largest cost.  group_of[i] receives the group of the
 * i-th ingress node (in node order); group_cost[g] the cost of group g.
 * Host only. */
int fhe_autohe(const fhe_graph_desc* g, uint32_t* group_of, uint32_t group_of_cap,
               uint32_t* group_cost, uint32_t group_cost_cap, uint32_t* n_groups);

/* Alg. autoHE then Alg. parameterise on a library graph: the ring degree and
 * coefficient-modulus bit list one parameter set needs to evaluate the whole
 * graph (the largest cost over its parameter groups; a graph whose groups
 * should get separate parameter sets uses fhe_autohe instead).  Host only. */
int fhe_autoparam(const fhe_graph* g, uint32_t log_scale, double special_mult,
                  uint32_t* N, uint32_t* bits, uint32_t bits_cap, uint32_t* n_bits);

/* Prime chain for (N, bits): q > 2^b, q = 1 mod 2N, increasing per size.
 * out receives n_bits primes (last = special prime).  Host only. */
int fhe_prime_chain(uint32_t N, const uint32_t* bits, uint32_t n_bits, uint64_t* out);

/* Discrete-Gaussian cumulative table used by the samplers (38 thresholds,
 * support [-19, 19], sigma 3.2).  Host only. */
int fhe_gauss_table(uint64_t* out38);

/* ---- context ------------------------------------------------------------ */

/* Build the context on the current CUDA device: primes, NTT tables and
 * encoder tables resident in HBM.  The NTT schedule (radix of the register
 * passes, threads per block, one- or two-pass, fused global I/O) is autotuned
 * here by timing each candidate on a rescale of 64 ciphertexts, and again
 * separately for the key-switching digit transforms (whose epilogue holds the
 * key inner product) on that step alone; the environment variable
 * FHE_NTT_VARIANT=0..8 fixes both instead (and FHE_NTT_VARIANT_KS, when set
 * with it, the key-switching one).  Schedule 6 splits each key-switching
 * digit transform over two blocks (one per output half, two blocks per SM);
 * schedule 7 runs the key-switching inner-product step on a cluster of four
 * blocks per (ciphertext, target prime), one per quarter of the
 * coefficients, with the accumulators in shared memory (N >= 256); the
 * other transforms run as schedule 5 under either.  Schedule 8 (1024 <= N
 * <= 16384, else schedule 5) runs each transform on N/32 threads: the first
 * log2 N - 10 stages block-wide, then each warp a 1024-point sub-transform
 * with warp-level synchronisation only.  bits: coefficient-modulus bit sizes, the
 * last one being the special prime; log_scale: scale 2^log_scale.
 * N must be a power of two in [16, 65536]; above 16384 only the two-pass
 * NTT schedules exist and the grouped (uneven-level) calls are refused. */
int fhe_ctx_create(uint32_t N, const uint32_t* bits, uint32_t n_bits,
                   uint32_t log_scale, fhe_ctx** out);
/* A fork shares the parent's tables and keys (resident once per parameter
 * set) and owns only its workspace, so calls on a parent and its forks may
 * run concurrently on different streams.  Forks of a fork fork the parent.
 * The parent must outlive its forks; keys must be generated on the parent
 * before forking (a fork copies the key pointers at fork time).  Serving
 * infrastructure: the paper has no counterpart. */
int fhe_ctx_fork(fhe_ctx* parent, fhe_ctx** out);
int fhe_ctx_destroy(fhe_ctx* ctx);
int fhe_ctx_query(const fhe_ctx* ctx, fhe_ctx_info* out);

/* Secret key s (ternary), public key and relinearisation keys (per-prime
 * digits, special prime P), sampled on the device from `seed`; resident in
 * HBM until the context is destroyed.  Synchronises `stream` at the end. */
int fhe_keygen(fhe_ctx* ctx, uint64_t seed, void* stream);

/* Device copy of the secret key (NTT form) [L_top + 1][N], for tests. */
int fhe_export_secret(fhe_ctx* ctx, uint64_t* d_out, void* stream);

/* ---- encode / encrypt / decrypt / decode -------------------------------- */

/* CKKS canonical-embedding encode: d_slots [n_ct][N/2] real -> plaintext
 * [n_ct][level][N] (NTT form); m_k = round(scale * sigma^{-1}(z)_k), half
 * away from zero.  The inverse DFT runs in 128-bit fixed point (64
 * fractional bits); the unrounded coefficients are within 2^-40 of exact.
 * Requires |slot| * scale < 2^61 (coefficients beyond that do not fit the
 * first prime in any case); larger inputs give unspecified coefficients. */
int fhe_encode(fhe_ctx* ctx, const double* d_slots, uint32_t n_ct, uint32_t level,
               double scale, uint64_t* d_pt, void* stream);

/* Public-key encryption at the top level: ct = (u pk0 + e0 + m, u pk1 + e1),
 * u ternary and e0, e1 Gaussian drawn from (keygen seed, ct id), ct id =
 * first_ct_id + k.  d_pt [n_ct][L_top][N] -> d_ct [n_ct][2][L_top][N]. */
int fhe_encrypt(fhe_ctx* ctx, const uint64_t* d_pt, uint32_t n_ct, uint64_t first_ct_id,
                uint64_t* d_ct, void* stream);

/* fhe_encode followed by fhe_encrypt in one pass: the encoded integer
 * coefficients join the first noise polynomial before its transform
 * (NTT(e0) + NTT(m) = NTT(e0 + m)), so no plaintext buffer or plaintext
 * transform is needed.  Same ciphertexts as the two calls. */
int fhe_encode_encrypt(fhe_ctx* ctx, const double* d_slots, uint32_t n_ct, double scale, uint64_t first_ct_id,
                       uint64_t* d_ct, void* stream);

/* Decrypt at `level`: m = c0 + c1 s, dropped to q_0, centred lift -> d_m
 * int64 [n_ct][N] (coefficient form). */
int fhe_decrypt(fhe_ctx* ctx, const uint64_t* d_ct, uint32_t n_ct, uint32_t level,
                int64_t* d_m, void* stream);

/* Decode: d_m int64 [n_ct][N] -> d_slots [n_ct][N/2] real parts, divided by
 * scale (FP64 FFT). */
int fhe_decode(fhe_ctx* ctx, const int64_t* d_m, uint32_t n_ct, double scale,
               double* d_slots, void* stream);

/* ---- rotations (slot rotation by a Galois automorphism) ------------------
 * Needed by slot-packed layouts (the paper's kernel masquerading, Sec. 3.2,
 * rotates ciphertexts to line pixels up with kernel positions).  Rotation
 * by r moves slot j + r to slot j (left), via X -> X^k, k = 5^r mod 2N, and a
 * key switch from s(X^k) back to s with a rotation key. */

/* Generate (once per parameter set, on the parent context) the rotation keys
 * for the given slot steps; each is resident like the relinearisation key
 * (L_top x 2 x (L_top + 1) x N x 16 bytes).  Keys already present are kept.
 * Sampling: domains 9 (uniform) and 10 (noise), object (k << 8) | digit.
 * Synchronises `stream`. */
int fhe_galois_keygen(fhe_ctx* ctx, const int32_t* steps, uint32_t n_steps, void* stream);

/* d_out [n_ct][2][level][N] = rotation of d_ct by `step` slots (NTT form).
 * FHE_ENOKEY if the rotation key of that step has not been generated. */
int fhe_rotate(fhe_ctx* ctx, const uint64_t* d_ct, uint32_t n_ct, uint32_t level, int32_t step, uint64_t* d_out,
               void* stream);

/* dst[r][c] = src_flat[index[r * cols + c]] (0 where the index is negative),
 * doubles, device memory: the client-side re-packing of decoded slots between
 * parameter groups (e.g. packed conv outputs -> one feature per ciphertext). */
int fhe_gather_slots(const double* d_src, const int64_t* d_index, uint32_t rows, uint32_t cols, double* d_dst,
                     void* stream);

/* ---- layout conversion (parity export / import) ------------------------- */

/* n_poly residue polynomials [n_poly][rows][N]: rows-th row r belongs to
 * prime index r (0..L_top, L_top = P).  forward = coefficient -> NTT form. */
int fhe_ntt(fhe_ctx* ctx, uint64_t* d_poly, uint32_t n_poly, uint32_t rows, int forward, void* stream);

/* ciphertexts [n_ct][2][level][N]: NTT form -> coefficient form (to_coeff = 1)
 * or back (to_coeff = 0); in and out may alias. */
int fhe_ct_convert(fhe_ctx* ctx, const uint64_t* d_in, uint32_t n_ct, uint32_t level,
                   int to_coeff, uint64_t* d_out, void* stream);

/* ---- homomorphic operations (batched; all at one level) ----------------- */

/* d_out = d_a + d_b */
int fhe_add(fhe_ctx* ctx, const uint64_t* d_a, const uint64_t* d_b, uint32_t n_ct, uint32_t level,
            uint64_t* d_out, void* stream);

/* tensor: d_out [n_ct][3][level][N] = (a0 b0, a0 b1 + a1 b0, a1 b1) */
int fhe_tensor(fhe_ctx* ctx, const uint64_t* d_a, const uint64_t* d_b, uint32_t n_ct, uint32_t level,
               uint64_t* d_out, void* stream);

/* relinearise: d3 [n_ct][3][level][N] -> d_out [n_ct][2][level][N] by RNS key
 * switching of the third component (per-prime digits, ModDown by P). */
int fhe_relinearise(fhe_ctx* ctx, const uint64_t* d3, uint32_t n_ct, uint32_t level,
                    uint64_t* d_out, void* stream);

/* Same result as fhe_relinearise, for callers that cannot allocate device
 * memory during the call (for instance a serving loop whose device memory
 * belongs to another allocator, or code that must not wait for the
 * device-wide synchronisation a workspace cudaMalloc/cudaFree can cause).
 * The paper has no counterpart: it is an allocation policy of this library.
 * Scratch comes from a fixed 16 MiB device array that every GPU loading the
 * library holds until exit; the call itself allocates and frees nothing.
 * The first call on a device (with the context's device current) looks up
 * that array's device address; under CUDA's lazy module loading (the
 * default) this is also when the library's module is loaded on that device
 * and the array is reserved, so that first call can allocate device memory
 * and fail with FHE_ENOMEM if another allocator already holds all of it.
 * Make one warm-up call per device before handing device memory to another
 * allocator and before any stream capture.  Batches needing more
 * scratch than 16 MiB ((L + 2(L+1) + 2) N 8 bytes per ciphertext, aligned)
 * return FHE_EINVAL.  All calls share the array: calls that overlap on the
 * GPU race and must be serialised by the caller. */
int fhe_relinearise_noalloc(fhe_ctx* ctx, const uint64_t* d3, uint32_t n_ct, uint32_t level,
                            uint64_t* d_out, void* stream);

/* rescale: d_in [n_ct][comps][level][N] -> d_out [n_ct][comps][level-1][N],
 * division by q_{level-1} with the centred remainder. */
int fhe_rescale(fhe_ctx* ctx, const uint64_t* d_in, uint32_t n_ct, uint32_t comps, uint32_t level,
                uint64_t* d_out, void* stream);

/* ct-mult + relinearise + rescale for n_ct pairs at `level`:
 * d_out [n_ct][2][level-1][N] = rescale(relin(a (x) b)).  ModDown and the
 * rescale share their forward transforms (NTT([v] P^-1 + [r]) per output
 * row, the transforms being linear); both centred roundings are those of
 * the separate steps, so the words equal fhe_relinearise then fhe_rescale.
 * The tensor product is not stored: each step recomputes the component it
 * needs from d_a and d_b.  d_out may overlap d_a or d_b (the tensor is then
 * formed in the workspace first). */
int fhe_mul_relin_rescale(fhe_ctx* ctx, const uint64_t* d_a, const uint64_t* d_b, uint32_t n_ct,
                          uint32_t level, uint64_t* d_out, void* stream);

/* One batch of ciphertext pairs at one level (for fhe_mul_relin_rescale_levels). */
typedef struct {
    const uint64_t* d_a;     /* [n_ct][2][level][N] */
    const uint64_t* d_b;     /* [n_ct][2][level][N] */
    uint64_t* d_out;         /* [n_ct][2][level-1][N] */
    uint32_t n_ct;
    uint32_t level;          /* 2 .. L_top */
} fhe_level_batch;

/* ct-mult + relinearise + rescale for ciphertexts at uneven levels in ONE
 * persistent kernel launch (plus a memset of its work queue): one block per
 * SM takes transform units from a device queue -- digit inverse transforms,
 * key inner products, inverse transforms of P's residues, then ModDown
 * merged with the rescale -- for every ciphertext of every batch; a unit
 * waits (bounded, about a second; FHE_ETIMEOUT if it gives up) for its
 * ciphertext's previous step, and the tensor product is recomputed from the
 * factors where needed instead of being stored.  Capturable in a CUDA graph
 * (after a first call has sized the workspace).  N <= 16384.  Up to 8
 * batches per launch (more are processed 8 at a time).  Same results as
 * fhe_mul_relin_rescale per batch.  FHE_PERSISTENT=0 in the environment
 * runs the same steps as six separate launches instead, for comparisons. */
int fhe_mul_relin_rescale_levels(fhe_ctx* ctx, const fhe_level_batch* batches, uint32_t n_batches, void* stream);

/* multiply by integer constants: ct_k *= C_k (one signed constant per
 * ciphertext, host array) ; and add integer constants to the constant term. */
int fhe_mul_const(fhe_ctx* ctx, const uint64_t* d_in, const int64_t* h_c, uint32_t n_ct, uint32_t level,
                  uint64_t* d_out, void* stream);
int fhe_add_const(fhe_ctx* ctx, uint64_t* d_ct, const int64_t* h_c, uint32_t n_ct, uint32_t level,
                  void* stream);

/* ---- graphs ------------------------------------------------------------- */

/* Copy a graph description (weights included) into a library-owned graph. */
int fhe_graph_create(const fhe_graph_desc* desc, fhe_graph** out);
int fhe_graph_destroy(fhe_graph* g);

/* Number of ciphertexts each OUTPUT node produces and their level, once the
 * graph is evaluated on a context whose inputs enter at L_top. */
int fhe_graph_outputs(fhe_ctx* ctx, const fhe_graph* g, uint32_t* n_out_cts, uint32_t* out_level);

/* Evaluate the graph (Alg. firing): d_in[i] holds the ciphertexts of the
 * i-th INPUT node ([n][2][L_top][N], scale 2^log_scale); the outputs of all
 * OUTPUT nodes, in node order, are written to d_out [n_out][2][out_level][N]
 * with one fhe_ct_meta each. */
int fhe_eval_graph(fhe_ctx* ctx, const fhe_graph* g, const uint64_t* const* d_in, uint32_t n_inputs,
                   uint64_t* d_out, fhe_ct_meta* out_meta, uint32_t out_cap, void* stream);

/* One encrypted-inference request of a served batch (Sec. 2.3 client/server
 * model; the batching itself has no counterpart in the paper).  x holds the
 * request's samples, one row per ciphertext of the graph's INPUT node
 * ([n_in] rows of x_stride doubles, the first n_samples used); y receives the
 * decoded outputs ([n_out] rows of y_stride doubles).  x and y may be device
 * or host memory (host memory should be pinned for the call to stay
 * asynchronous); the caller owns both. */
typedef struct {
    const double* x;
    uint32_t n_samples;
    uint32_t x_stride;
    double* y;
    uint32_t y_stride;
} fhe_request;

/* Serve a batch of requests through a graph with exactly one INPUT node:
 * request k occupies the slot range after requests 0..k-1 (at most N/2
 * samples in total, else FHE_EINVAL; unused slots hold 0), then, all on
 * `stream`: the rows are gathered into the slots, encoded and encrypted at
 * the top level with scale 2^log_scale and ct ids first_ct_id + i, the graph
 * is evaluated, the outputs decrypted and decoded, and each request's columns
 * copied to its y.  Buffers come from a context-owned batch area (grown on
 * demand, separate from the workspace), so forks of one parameter set can
 * serve concurrent batches on their own streams.  Results are those of
 * fhe_encode_encrypt + fhe_eval_graph + fhe_decrypt + fhe_decode on the packed
 * slots. */
int fhe_eval_batch(fhe_ctx* ctx, const fhe_graph* g, const fhe_request* reqs, uint32_t n_reqs,
                   uint64_t first_ct_id, void* stream);

/* ---- measurement (no counterpart in the paper) ----------------------------
 * fhe_profile_begin: from now on, every launch of the kernel family `family`
 * made through this context ("keyswitch_modup_mac", "mac", "rescale_ntt", ...,
 * the names fhe_profile_families lists) is bracketed by CUDA events recorded
 * on its own stream (up to max_launches launches).  fhe_profile_end
 * synchronises those events and returns the summed device time in ms, the
 * number of launches and how many of them were timed; profiling then stops. */
int fhe_profile_begin(fhe_ctx* ctx, const char* family, uint32_t max_launches);
int fhe_profile_end(fhe_ctx* ctx, double* total_ms, uint64_t* launches, uint64_t* timed);
/* Comma-separated list of the kernel family names (static string). */
const char* fhe_profile_families(void);
/* Number of kernels this library has launched in the process so far. */
int fhe_launch_count(uint64_t* out);
/* Health hook (no counterpart in the paper): reads and clears the device
 * fault flags of the current device.  Bit 0: a tensor-core layer MAC block
 * gave up waiting for its matrix products (its waits are bounded, well under a
 * second) and left its outputs unwritten.  Synchronises the device; *out = 0
 * when no wait gave up since the last call. */
int fhe_device_faults(uint32_t* out);

/* Integer-pipe ceiling microbenchmark (no counterpart in the paper; the
 * denominators of the ALU roofline).  Enqueues one kernel of `blocks` x
 * `threads` threads (threads a multiple of 32, at most 1024), each running
 * `iters` steps of 32 independent operations of one kind held in registers:
 *   0  32-bit multiply-add (IMAD)
 *   1  32 x 32 -> 64-bit multiply-add (IMAD.WIDE)
 *   2  high half of a 64 x 64-bit product
 *   3  Shoup butterfly of the fused transforms for primes below 2^58:
 *      T = a w - floor(a w' / 2^64) q, (X, Y) -> (X + T, X + 2q - T)
 *   4  the same butterfly in Harvey's form (X reduced below 2q first)
 * so blocks * threads * iters * 32 operations in all.  d_sink (device,
 * blocks * threads words, caller-owned) receives one word per thread.  Time
 * it with events on `stream`. */
int fhe_peak_launch(uint32_t kind, uint32_t blocks, uint32_t threads, uint32_t iters, uint64_t* d_sink,
                    void* stream);

/* Wait for `stream`, then report the context's health: FHE_ETIMEOUT if a
 * kernel launched through this context gave up a bounded device wait since
 * the last report (its outputs are then unspecified), else FHE_OK.  The
 * report clears the status.  Serving infrastructure: the paper has no
 * counterpart. */
int fhe_ctx_sync(fhe_ctx* ctx, void* stream);

/* Test hook (no counterpart in the paper): make a failure happen on purpose,
 * on the host's side of the device, without faulting anything.
 * FHE_INJECT_MAC_TC_WITHHOLD: the next tensor-core layer MAC launched through
 * this context issues none of its matrix products and shortens its waits to
 * about a millisecond, so every block's bounded wait runs out with no tensor
 * work in flight; the blocks free their tensor memory and return, the layer's
 * outputs are left unwritten, and the context reports FHE_ETIMEOUT.  The
 * context stays usable. */
#define FHE_INJECT_MAC_TC_WITHHOLD 1u
/* FHE_INJECT_PERSIST_STALL: in the next persistent uneven-level launch
 * (fhe_mul_relin_rescale_levels) through this context, the first phase's
 * units never report completion and the waits are shortened to about a
 * millisecond, so the second phase's bounded waits run out: the launch
 * aborts its remaining units, leaves the outputs unwritten, and the context
 * reports FHE_ETIMEOUT.  The context stays usable. */
#define FHE_INJECT_PERSIST_STALL 2u
int fhe_inject_fault(fhe_ctx* ctx, uint32_t kind);

const char* fhe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FHE_H */
