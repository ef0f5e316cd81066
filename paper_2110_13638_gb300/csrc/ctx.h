// ctx.h -- internal context of libfhe (not part of the C ABI).
#pragma once
#include <cstdint>
#include <string>
#include <map>
#include <vector>

#include <cuda_runtime.h>

#include "fhe_device.cuh"

struct fhe_ctx {
    uint32_t N = 0, logN = 0, L_top = 0, log_scale = 0;
    std::vector<u64> primes;       // q_0 .. q_{L_top-1}, P (index L_top)
    std::vector<PrimeC> pc;        // host copy of the per-prime constants
    double delta = 0.0;
    int device = 0;
    int ntt_variant = 0;           // NTT schedule (see ntt_variant_name), autotuned
    float ntt_variant_us[16] = {};   // autotuner: us per transform per variant
    int ntt_variant_ks = 0;        // schedule of the key-switching inner-product transforms
    bool ntt_forced = false;       // the schedules were fixed by FHE_NTT_VARIANT (no launch-time change)
    int sms = 0;                   // SMs of the device
    float ntt_variant_ks_us[16] = {};
    u64* d_ntt2 = nullptr;         // two-pass intermediate (allocated with the context)
    size_t ntt2_words = 0;

    // resident tables
    PrimeC* d_pc = nullptr;
    ulonglong2* d_tw_fwd = nullptr;
    ulonglong2* d_tw_inv = nullptr;
    ulonglong2* d_tw_fwd_wl = nullptr;   // warp-local layouts (NttTables::tw_fwd_wl)
    ulonglong2* d_tw_inv_wl = nullptr;
    u64* d_cdt = nullptr;          // 38 Gaussian thresholds
    double4* d_enc_tw = nullptr;   // [N/4] zeta^{-4k} as (re.hi, re.lo, im.hi, im.lo)
    double4* d_enc_twist = nullptr;// [N/2] zeta^{-k}
    // the same roots as fixed point for the encoder: [k][0] = re, [k][1] = im,
    // each (low word, high word | sign << 63), magnitude scaled by 2^126
    ulonglong2* d_enc_tw_q = nullptr;    // [N/4][2]
    ulonglong2* d_enc_twist_q = nullptr; // [N/2][2]
    uint32_t* d_slot_of = nullptr; // [N/2] FFT position l -> slot j

    // keys (NTT form)
    bool has_keys = false;
    uint64_t seed = 0;
    u64* d_s = nullptr;            // [L_top + 1][N]
    u64* d_pk = nullptr;           // [2][L_top][N]
    u64* d_pks = nullptr;          // [2][L_top][N] Shoup quotients floor(pk 2^64 / q) of d_pk
    ulonglong2* d_ksk = nullptr;   // [L_top][2][L_top + 1][N] (key word, Shoup quotient)
    std::map<u64, ulonglong2*> galois;   // Galois element k -> rotation key (same layout); forks use the parent's
    size_t key_bytes = 0;

    // a fork shares tables and keys with its parent (which must outlive it)
    // and owns only its workspace and two-pass scratch
    fhe_ctx* parent = nullptr;

    // call workspace (grows on demand)
    void* ws = nullptr;
    size_t ws_bytes = 0;
    void* bb = nullptr;            // fhe_eval_batch's slots / ciphertext area (own per fork)
    size_t bb_bytes = 0;

    // health: a host-mapped word that a kernel sets when one of its bounded
    // waits gives up (read and cleared by fhe_ctx_sync and the graph calls);
    // one per context, forks included
    unsigned int* h_status = nullptr;
    unsigned int* d_status = nullptr;      // device address of h_status
    mutable int inject = 0;                // test hook (fhe_inject_fault), consumed by the next launch it names

    // measurement hook: CUDA events around every launch of one kernel family
    mutable std::string prof_family;
    mutable std::vector<cudaEvent_t> prof_ev;   // pairs (start, stop)
    mutable size_t prof_used = 0;
    mutable uint64_t prof_launches = 0;

    NttTables tabs() const
    {
        NttTables t;
        t.tw_fwd = d_tw_fwd;
        t.tw_inv = d_tw_inv;
        t.tw_fwd_wl = d_tw_fwd_wl;
        t.tw_inv_wl = d_tw_inv_wl;
        t.pc = d_pc;
        t.logN = (int)logN;
        return t;
    }
};

struct fhe_graph_node {
    uint32_t kind = 0;
    uint32_t n_out = 0;
    std::vector<uint32_t> row_ptr, col_idx;
    std::vector<double> weight, bias;
    double coeffs[4] = {0, 0, 0, 0};
    uint32_t degree = 3;       // POLY / RELU (RELU: coefficients of Eq. relu_approximate, degree 2)
    uint32_t conv[6] = {0, 0, 0, 0, 0, 0};   // CONV_PACKED: H, W, k, stride, images, slot stride
    std::vector<double> poly;  // POLY of degree > 3: a_0 .. a_degree
};

// device constants of one node at its planned level (built on first use)
struct fhe_node_const {
    uint32_t L = 0;            // input level the constants were made for
    double s_in = 0.0;         // input nominal scale they were made for
    void* buf = nullptr;       // one device allocation holding the arrays below
    uint32_t* row_ptr = nullptr;
    uint32_t* col = nullptr;
    u64* W = nullptr;          // LINEAR: weight residues, tile order (see k_linear_mac_tiled)
    uint4* tiles = nullptr;    // LINEAR: row tiles {col_off, K, n_rows, w_off}
    uint32_t* tile_rows = nullptr;
    uint32_t n_tiles = 0;
    uint32_t max_tile_rows = 0;   // LINEAR: the most rows a tile holds
    u64* bias = nullptr;       // LINEAR: [n_out][L-1] bias residues
    struct TcPart {            // LINEAR, dense: one limb count of the tensor-core MAC
        uint16_t* W = nullptr; // weight limbs (see k_linear_mac_tc)
        uint32_t* rows = nullptr;
        uint32_t tiles = 0;
        uint64_t mask = 0;     // its residues
    } tc[2];                   // five limbs, eight limbs
    uint32_t tc_K = 0;
    bool tc_on = false;        // the setting the constants were made for
    u64* c3 = nullptr;         // POLY: constant residues (shared by all ciphertexts)
    u64* c2 = nullptr;
    u64* c1 = nullptr;
    u64* c0 = nullptr;
    u64* c3s = nullptr;        // POLY: Shoup quotients of c3, c2, c1
    u64* c2s = nullptr;
    u64* c1s = nullptr;
    u64* cpow = nullptr;       // POLY degree > 3: residues of C_1..C_d at l* primes, then C_0 ([d + 1][l*])
    u64* pt = nullptr;         // CONV_PACKED: mask-and-kernel plaintexts [F][k^2][L][N] (NTT form)
    u64* bias_pt = nullptr;    // CONV_PACKED: bias plaintexts [F][L-1][N]
};

struct fhe_graph {
    std::vector<fhe_graph_node> nodes;
    std::vector<uint32_t> esrc, edst;
    const fhe_ctx* cache_ctx = nullptr;
    std::vector<fhe_node_const> cache;
};

namespace fhe {

// every kernel launch of the library goes through this scope: it counts the
// launch and, when the context profiles that family, brackets it with events
struct LaunchScope {
    const fhe_ctx* c;
    cudaStream_t st;
    long idx = -1;
    LaunchScope(const fhe_ctx* c, const char* family, cudaStream_t st);
    ~LaunchScope();
};
uint64_t launch_count();

// error reporting (thread-local message)
int fail(int code, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);

// ---- workspace arena -----------------------------------------------------
struct Arena {
    char* base = nullptr;
    size_t cap = 0, used = 0;
    void* take(size_t bytes)
    {
        size_t a = (used + 255) & ~(size_t)255;
        if (a + bytes > cap) return nullptr;
        used = a + bytes;
        return base + a;
    }
};
int ws_reserve(fhe_ctx* c, size_t bytes, Arena* a);
// Reads and clears the context's status word without synchronising:
// FHE_ETIMEOUT if a kernel launched through this context gave up one of its
// bounded waits and has finished since the word was last read, else FHE_OK.
int status_take(const fhe_ctx* c);
inline size_t arena_need(std::initializer_list<size_t> parts)
{
    size_t s = 0;
    for (size_t p : parts) s += ((p + 255) & ~(size_t)255);
    return s;
}

// ---- per-level constants (host-computed, passed by value) ------------------
struct DivC {           // division by one prime p into primes q_0..q_{n-1}
    u64 p, p_half;
    u64 inv[32], invs[32];    // p^{-1} mod q_i and its Shoup quotient
    u64 pmod[32];             // p mod q_i
};
DivC make_divc(const fhe_ctx* c, uint32_t p_index, uint32_t n_targets);
void k_modup_mac_step(const fhe_ctx* c, const u64* d3, const u64* D, const ulonglong2* ksk, u64* acc, uint32_t n_ct,
                      uint32_t L, cudaStream_t st);

// ---- kernels (kernels.cu); all enqueue on `st` -------------------------
void k_ntt_rows(const fhe_ctx* c, u64* d, uint32_t n_poly, uint32_t rows, const uint8_t* row_prime,
                bool forward, cudaStream_t st);
void k_ct_to_coeff(const fhe_ctx* c, const u64* in, u64* out, uint32_t n_ct, uint32_t comps, uint32_t L,
                   bool to_coeff, cudaStream_t st);
void k_add(const fhe_ctx* c, const u64* a, const u64* b, u64* out, uint32_t n_ct, uint32_t comps, uint32_t L,
           cudaStream_t st);
void k_tensor(const fhe_ctx* c, const u64* a, const u64* b, u64* out3, uint32_t n_ct, uint32_t L, cudaStream_t st);
// scratch: relin_scratch_bytes(n_ct, L)
size_t relin_scratch_bytes(const fhe_ctx* c, uint32_t n_ct, uint32_t L);
// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device (once per kernel, device and size; thread-safe).
void ensure_smem(const void* kernel, size_t bytes);

// key: the relinearisation key unless another key of the same layout is given;
// single_pass: no two-pass schedule (scratch is then the only memory used
// besides d3 and out2)
void k_relin(const fhe_ctx* c, const u64* d3, u64* out2, uint32_t n_ct, uint32_t L, void* scratch, cudaStream_t st,
             const ulonglong2* key = nullptr, bool single_pass = false);
// rotation key for Galois element k into `key` ([L_top][2][L_top + 1][N])
void k_galois_keygen(fhe_ctx* c, u64 k, ulonglong2* key, cudaStream_t st);
// d3 = (c0(X^k), 0, c1(X^k)) of ciphertexts [n][2][L][N] in NTT form
void k_automorph(const fhe_ctx* c, const u64* ct, u64* d3, uint32_t n_ct, uint32_t L, u64 k, cudaStream_t st);
// Galois element of a slot rotation by `step`; rotation keys of the given steps
u64 galois_element_of(const fhe_ctx* c, int64_t step);
int galois_keys_for(fhe_ctx* root, const std::vector<int64_t>& steps, cudaStream_t st);
// packed convolution: Y[f * n + i] (+)= X[i] * PT[f][p] slot-wise (NTT form, both components)
void k_plain_mac(const fhe_ctx* c, u64* Y, const u64* X, const u64* PT, uint32_t F, uint32_t n, uint32_t L,
                 uint32_t p, uint32_t k2, bool accumulate, cudaStream_t st);
// comp 0 of out[f * n + i] += BIAS[f] (level L1)
void k_add_plain(const fhe_ctx* c, u64* out, const u64* bias, uint32_t F, uint32_t n, uint32_t L1, cudaStream_t st);
void k_gather_slots(const double* src, const int64_t* index, size_t total, double* dst, cudaStream_t st);
// relinearise then rescale, fused (ModDown's and the rescale's forward
// transforms merged; word for word the two steps in sequence):
// out [n][2][L-1][N] = rescale(relin(d3) + E) (+ addc on comp 0, as k_rescale),
// E = x2 c2 + x c1 when ex is given (fields may be null)
struct KsExtra {
    const u64* x2;      // [n][2][L][N] (level of the relinearisation) or null
    const u64* c2;      // [L] device residues
    const u64* c2s;     // their Shoup quotients
    const u64* x;       // [n][2][Lx][N], its first L residues used, or null
    const u64* c1;      // [L] device residues
    const u64* c1s;     // their Shoup quotients
    int Lx;
};
size_t relin_rescale_scratch_bytes(const fhe_ctx* c, uint32_t n_ct, uint32_t L);
void k_relin_rescale(const fhe_ctx* c, const u64* d3, u64* out, uint32_t n_ct, uint32_t L, void* scratch,
                     cudaStream_t st, const KsExtra* ex = nullptr, const u64* addc = nullptr,
                     uint32_t addc_stride = 0);
// the same for the tensor product of a and b ([n][2][L][N] each, NTT form,
// reduced) without storing it (k_relin_tensor.cu); same scratch
void k_mul_relin_rescale(const fhe_ctx* c, const u64* a, const u64* b, u64* out, uint32_t n_ct, uint32_t L,
                         void* scratch, cudaStream_t st);
// scratch: rescale_scratch_bytes; addc: optional constants (device residues,
// addc[ct * addc_stride + i]) added to comp 0 of the result
size_t rescale_scratch_bytes(const fhe_ctx* c, uint32_t n_ct, uint32_t comps);
void k_rescale(const fhe_ctx* c, const u64* in, u64* out, uint32_t n_ct, uint32_t comps, uint32_t L,
               const u64* addc, uint32_t addc_stride, void* scratch, cudaStream_t st, const u64* mulc = nullptr,
               const u64* mulcs = nullptr);
// (x2 (x) rescale(x * C)) into out3 [n][3][L-1][N]: the rescale's forward
// transforms with the tensor product in their epilogue (x at level L, x2 at
// L-1; C: per-residue constants with their Shoup quotients)
size_t rescale_tensor_scratch_bytes(const fhe_ctx* c, uint32_t n_ct, uint32_t L);
void k_rescale_tensor(const fhe_ctx* c, const u64* x, const u64* mulc, const u64* mulcs, const u64* x2, u64* out3,
                      uint32_t n_ct, uint32_t L, void* scratch, cudaStream_t st);
// polynomial activation: t1 (+)= x2 * c2 + (first L1 residues of x) * c1
// (accumulate: add to t1; else overwrite it)
void k_poly_combine(const fhe_ctx* c, u64* t1, const u64* x2, const u64* x, uint32_t n_ct, uint32_t L1, uint32_t Lx,
                    const u64* c2, const u64* c1, cudaStream_t st, bool accumulate = true);
// constants C (device residues cres[ct * cstride + r]) multiply every component;
// reads residues r < L_out of an input stored with L_in residues
void k_mul_const(const fhe_ctx* c, const u64* in, u64* out, uint32_t n_ct, uint32_t comps, uint32_t L_in,
                 uint32_t L_out, const u64* cres, uint32_t cstride, cudaStream_t st);
void k_add_const(const fhe_ctx* c, u64* ct, uint32_t n_ct, uint32_t L, const u64* cres, uint32_t cstride,
                 cudaStream_t st);
// gather-MAC: Y[o][k][r] = sum_e W[e][r] X[col[e]][k][r] over CSR row o (all at level L)
// tiled gather-MAC (rows sharing a column list computed together)
constexpr int kMacTile = 6;
// primes below this bound store MAC weights as 21-bit limbs (wL | wH << 32)
constexpr unsigned long long kLimbPrimeBound = 1ull << 42;
// skip_mask: residues r with bit r set are left to the tensor-core MAC;
// max_tile_rows: the most rows any tile holds (five or fewer: a cheaper kernel)
void k_linear_mac_tiled(const fhe_ctx* c, const u64* X, const uint4* tiles, uint32_t n_tiles, const uint32_t* rows,
                        const uint32_t* col, const u64* W, uint32_t L, u64* Y, cudaStream_t st,
                        uint64_t skip_mask = 0, uint32_t max_tile_rows = kMacTile);
// tensor-core MAC of a dense layer (every row over the same K input columns),
// residues r with bit r of mask set: five limbs for primes below 2^41 (tiles
// of kMacTcRows rows), eight below 2^61 (tiles of kMacTcRows8 rows):
//   Wl = bf16 weight limbs [residue of the mask][tile][chunk][limb][rows x 32, core-matrix order],
//   rows[tile * tile rows + o] = output row (0xFFFFFFFF: none)
constexpr int kMacTcRows = 48;
constexpr int kMacTcRows8 = 32;
constexpr int kMacTcChunk = 32;
constexpr unsigned long long kMacTcPrimeBound5 = 1ull << 41;
constexpr unsigned long long kMacTcPrimeBound8 = 1ull << 61;
int k_linear_mac_tc(const fhe_ctx* c, int limbs, const u64* X, const uint32_t* col, uint32_t K, const uint16_t* Wl,
                    const uint32_t* rows, uint32_t n_tiles, uint64_t mask, uint32_t L, u64* Y, cudaStream_t st);
// reads and clears the tensor-core MAC's fault flag (a wait that gave up); synchronous
uint32_t mac_tc_fault_take();

// ct-mult + relinearise + rescale over batches at different levels (<= 8 batches)
struct LevelBatch {
    const u64* a;
    const u64* b;
    u64* out;
    uint32_t n, L;
};
size_t level_groups_scratch_bytes(const fhe_ctx* c, const LevelBatch* g, int ng);
void k_mul_relin_rescale_groups(const fhe_ctx* c, const LevelBatch* g, int ng, void* scratch, cudaStream_t st);
// the same in one persistent launch (N <= 16384; plus one memset of its queue)
size_t persist_scratch_bytes(const fhe_ctx* c, const LevelBatch* g, int ng);
int k_mul_relin_rescale_persistent(const fhe_ctx* c, const LevelBatch* g, int ng, void* scratch, cudaStream_t st);

void k_keygen(fhe_ctx* c, cudaStream_t st);
size_t encrypt_scratch_bytes(const fhe_ctx* c, uint32_t n_ct);
void k_encrypt(const fhe_ctx* c, const u64* pt, uint32_t n_ct, uint64_t first_id, u64* ct, void* scratch,
               cudaStream_t st);
void k_decrypt(const fhe_ctx* c, const u64* ct, uint32_t n_ct, uint32_t L, i64* m, cudaStream_t st);
size_t encode_scratch_bytes(const fhe_ctx* c, uint32_t n_ct);
void k_encode(const fhe_ctx* c, const double* slots, uint32_t n_ct, uint32_t L, double scale, u64* pt,
              void* scratch, cudaStream_t st);
void k_decode(const fhe_ctx* c, const i64* m, uint32_t n_ct, double scale, double* slots, cudaStream_t st);
void encode_coefficients(const fhe_ctx* c, const double* slots, uint32_t n_ct, double scale, i64* m, cudaStream_t st);
size_t encode_encrypt_scratch_bytes(const fhe_ctx* c, uint32_t n_ct);
void k_encode_encrypt(const fhe_ctx* c, const double* slots, uint32_t n_ct, double scale, uint64_t first_id, u64* ct,
                      void* scratch, cudaStream_t st);

uint64_t stream_key(uint64_t seed, uint64_t domain, uint64_t object);
const char* ntt_variant_name(int v);
// the ModUp cluster schedule (7) handles this ring
bool modup_cluster_fits(const fhe_ctx* c);
constexpr int kNttVariants = 9;   // schedules 6 and 7 apply to the key-switching digit transforms only
inline bool ntt_two_pass(int v) { return v == 2 || v == 3; }
inline bool ntt_ks_only(int v) { return v == 6 || v == 7; }
// the warp-local schedule (8) needs 1024 <= N <= 16384; below, schedule 5 stands in
inline bool ntt_wl_fits(uint32_t logN) { return logN >= 10 && logN <= 14; }
constexpr uint32_t kMaxSinglePassN = 16384;   // one transform per block in shared memory

}  // namespace fhe
