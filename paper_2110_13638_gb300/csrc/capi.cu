// capi.cu -- the extern "C" entry points of libfhe (include/fhe.h): context
// and key management, batched homomorphic operations, and graph evaluation
// (the neuronal-firing traversal of arXiv 2110.13638, Sec. 3, Alg. firing /
// signal_carrier / get_inbound_signal / apply_signal / set_outbound_signals),
// whose node receptors launch the kernels of kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/fhe.h"
#include "ctx.h"
#include "host_math.h"

using namespace fhe;

static constexpr uint32_t kMaxLevelBatches = 8;

namespace fhe {

static thread_local std::string g_err;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

int cuda_check(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return FHE_OK;
    return fail(e == cudaErrorMemoryAllocation ? FHE_ENOMEM : FHE_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

int ws_reserve(fhe_ctx* c, size_t bytes, Arena* a)
{
    if (bytes == 0) bytes = 256;
    if (c->ws_bytes < bytes) {
        if (c->ws) {
            cudaDeviceSynchronize();
            cudaFree(c->ws);
            c->ws = nullptr;
            c->ws_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&c->ws, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_check(e, "workspace cudaMalloc");
        }
        c->ws_bytes = bytes;
    }
    a->base = (char*)c->ws;
    a->cap = c->ws_bytes;
    a->used = 0;
    return FHE_OK;
}

int status_take(const fhe_ctx* c)
{
    volatile unsigned int* h = c->h_status;
    if (!h || *h == 0) return FHE_OK;
    *h = 0;
    return fail(FHE_ETIMEOUT, "a kernel's bounded device wait gave up; its outputs were not written");
}

// llround of a double: round half away from zero (C semantics)
static int64_t dround(double x) { return (int64_t)std::llround(x); }

static u64 mod_signed(int64_t v, u64 q)
{
    if (v >= 0) return (u64)v % q;
    u64 r = (u64)(-(v + 1)) % q;            // |v| - 1 mod q
    r = (r + 1) % q;
    return r == 0 ? 0 : q - r;
}

}  // namespace fhe

#define CHECK_CTX(c)                                                         \
    do {                                                                     \
        if (!(c)) return fail(FHE_EINVAL, "null context");                  \
    } while (0)
#define CHECK_KEYS(c)                                                        \
    do {                                                                     \
        if (!(c)->has_keys) return fail(FHE_ENOKEY, "fhe_keygen has not run"); \
    } while (0)
#define CUDA_LAST(what)                                                      \
    do {                                                                     \
        cudaError_t _e = cudaGetLastError();                                 \
        if (_e != cudaSuccess) return cuda_check(_e, what);                  \
    } while (0)

// ---------------------------------------------------------------- rotation keys
namespace fhe {
u64 galois_element_of(const fhe_ctx* c, int64_t step)
{
    const int64_t half = c->N / 2;
    int64_t r = step % half;
    if (r < 0) r += half;
    u64 k = 1;
    for (int64_t i = 0; i < r; ++i) k = (k * 5) % (2ull * c->N);
    return k;
}

// generate the missing rotation keys of `steps` on the parent context (async on st)
int galois_keys_for(fhe_ctx* root, const std::vector<int64_t>& steps, cudaStream_t st)
{
    const size_t bytes = (size_t)root->L_top * 2 * (root->L_top + 1) * root->N * sizeof(ulonglong2);
    for (int64_t step : steps) {
        const u64 k = galois_element_of(root, step);
        if (k == 1 || root->galois.count(k)) continue;       // identity, or already there
        ulonglong2* key = nullptr;
        cudaError_t e = cudaMalloc((void**)&key, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_check(e, "rotation key allocation");
        }
        k_galois_keygen(root, k, key, st);
        root->galois[k] = key;
        root->key_bytes += bytes;
    }
    return FHE_OK;
}
}  // namespace fhe

extern "C" {

const char* fhe_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------- parameters
int fhe_parameterise(uint32_t cost, uint32_t log_scale, double special_mult, uint32_t* N, uint32_t* bits,
                     uint32_t bits_cap, uint32_t* n_bits)
{
    if (!N || !bits || !n_bits) return fail(FHE_EINVAL, "null output");
    std::vector<uint32_t> b;
    parameterise(cost, log_scale, special_mult, N, b);
    *n_bits = (uint32_t)b.size();
    if (b.size() > bits_cap) return fail(FHE_EINVAL, "bits_cap too small");
    for (size_t i = 0; i < b.size(); ++i) bits[i] = b[i];
    return FHE_OK;
}

int fhe_prime_chain(uint32_t N, const uint32_t* bits, uint32_t n_bits, uint64_t* out)
{
    if (!bits || !out || n_bits == 0) return fail(FHE_EINVAL, "bad arguments");
    if (N < 2 || (N & (N - 1))) return fail(FHE_EINVAL, "N must be a power of two");
    std::vector<u64> ch;
    if (!prime_chain(N, bits, n_bits, ch)) return fail(FHE_EINVAL, "bit size out of range [20, 61]");
    for (uint32_t i = 0; i < n_bits; ++i) out[i] = ch[i];
    return FHE_OK;
}

int fhe_gauss_table(uint64_t* out38)
{
    if (!out38) return fail(FHE_EINVAL, "null output");
    std::vector<u64> t = gauss_cdt();
    for (size_t i = 0; i < t.size(); ++i) out38[i] = t[i];
    return FHE_OK;
}

// Alg. autoHE_discover: largest accumulated cost from source s at every node;
// a node of the concern type (input / output) reached from another source
// restarts discovery as its own source with cost 0.
static uint32_t node_cost(const fhe_node_desc& nd)
{
    switch (nd.kind) {
    case FHE_NODE_LINEAR: return 1;
    case FHE_NODE_SQUARE: return 1;
    case FHE_NODE_POLY: {
        const uint32_t d = nd.degree == 0 ? 3 : nd.degree;
        if (d <= 3) return d == 1 ? 1 : 2;                  // affine: one rescale
        uint32_t lg = 0;
        while ((1u << lg) < d) ++lg;
        return lg + 1;                                      // powers, then the combining rescale
    }
    case FHE_NODE_RELU: return 2;
    case FHE_NODE_CONV_PACKED: return 1;
    default: return 0;
    }
}

static bool is_concern(uint32_t kind)
{
    return kind == FHE_NODE_INPUT || kind == FHE_NODE_OUTPUT || kind == FHE_NODE_ROTATE;
}

struct Discover {
    const fhe_graph_desc* g;
    std::vector<std::map<uint32_t, uint32_t>> sources;   // node -> {source: cost}
    std::vector<std::vector<uint32_t>> succ;
    int depth = 0;
    bool overflow = false;
    void run(uint32_t n, uint32_t s, uint32_t c)
    {
        if (++depth > 100000) { overflow = true; --depth; return; }
        auto& d = sources[n];
        if (s != n) {
            auto it = d.find(s);
            if (it == d.end() || it->second < c) d[s] = c;
        }
        if (is_concern(g->nodes[n].kind) && s != n) {
            run(n, n, 0);
        } else {
            for (uint32_t i : succ[n]) run(i, s, c + node_cost(g->nodes[i]));
        }
        --depth;
    }
};

int fhe_autohe(const fhe_graph_desc* g, uint32_t* group_of, uint32_t group_of_cap, uint32_t* group_cost,
               uint32_t group_cost_cap, uint32_t* n_groups)
{
    if (!g || !g->nodes || !n_groups) return fail(FHE_EINVAL, "null graph");
    Discover D;
    D.g = g;
    D.sources.resize(g->n_nodes);
    D.succ.resize(g->n_nodes);
    for (uint32_t e = 0; e < g->n_edges; ++e) {
        uint32_t a = g->edge_src[e], b = g->edge_dst[e];
        if (a >= g->n_nodes || b >= g->n_nodes) return fail(FHE_EINVAL, "edge out of range");
        auto& v = D.succ[a];
        if (std::find(v.begin(), v.end(), b) == v.end()) v.push_back(b);
    }
    std::vector<uint32_t> inputs;          // ingress nodes: INPUT and ROTATE
    for (uint32_t i = 0; i < g->n_nodes; ++i)
        if (g->nodes[i].kind == FHE_NODE_INPUT || g->nodes[i].kind == FHE_NODE_ROTATE) inputs.push_back(i);
    for (uint32_t i : inputs) D.run(i, i, 0);
    if (D.overflow) return fail(FHE_EINVAL, "graph traversal too deep (cycle without a concern node?)");
    std::map<uint32_t, uint32_t> gof;
    std::vector<uint32_t> gcost;
    for (uint32_t i : inputs) {
        if (!gof.count(i)) {
            gof[i] = (uint32_t)gcost.size();
            gcost.push_back(0);
        }
        for (uint32_t j = 0; j < g->n_nodes; ++j) {
            const auto& src = D.sources[j];
            if (!src.count(i)) continue;
            for (const auto& kv : src) {
                gof[kv.first] = gof[i];
                if (kv.second > gcost[gof[i]]) gcost[gof[i]] = kv.second;
            }
        }
    }
    *n_groups = (uint32_t)gcost.size();
    if (group_of) {
        if (inputs.size() > group_of_cap) return fail(FHE_EINVAL, "group_of_cap too small");
        for (size_t k = 0; k < inputs.size(); ++k) group_of[k] = gof[inputs[k]];
    }
    if (group_cost) {
        if (gcost.size() > group_cost_cap) return fail(FHE_EINVAL, "group_cost_cap too small");
        for (size_t k = 0; k < gcost.size(); ++k) group_cost[k] = gcost[k];
    }
    return FHE_OK;
}

int fhe_autoparam(const fhe_graph* g, uint32_t log_scale, double special_mult, uint32_t* N, uint32_t* bits,
                  uint32_t bits_cap, uint32_t* n_bits)
{
    if (!g) return fail(FHE_EINVAL, "null graph");
    std::vector<fhe_node_desc> nodes(g->nodes.size());
    uint32_t n_in = 0;
    for (size_t i = 0; i < g->nodes.size(); ++i) {
        std::memset(&nodes[i], 0, sizeof(fhe_node_desc));
        nodes[i].kind = g->nodes[i].kind;
        nodes[i].degree = g->nodes[i].degree;
        n_in += g->nodes[i].kind == FHE_NODE_INPUT || g->nodes[i].kind == FHE_NODE_ROTATE;
    }
    fhe_graph_desc d;
    d.n_nodes = (uint32_t)nodes.size();
    d.nodes = nodes.data();
    d.n_edges = (uint32_t)g->esrc.size();
    d.edge_src = g->esrc.data();
    d.edge_dst = g->edst.data();
    std::vector<uint32_t> gcost(std::max<uint32_t>(1u, n_in));
    uint32_t ng = 0;
    int rc = fhe_autohe(&d, nullptr, 0, gcost.data(), (uint32_t)gcost.size(), &ng);
    if (rc) return rc;
    if (ng == 0) return fail(FHE_EINVAL, "graph without INPUT nodes");
    uint32_t cost = 0;
    for (uint32_t k = 0; k < ng; ++k) cost = std::max(cost, gcost[k]);
    return fhe_parameterise(cost, log_scale, special_mult, N, bits, bits_cap, n_bits);
}


// ---------------------------------------------------------------- context
static void free_ctx(fhe_ctx* c)
{
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    cudaFreeHost(c->h_status);
    cudaFree(c->bb);
    if (c->parent) {            // shared tables and keys belong to the parent
        cudaFree(c->ws);
        cudaFree(c->d_ntt2);
        delete c;
        return;
    }
    cudaFree(c->d_pc);
    cudaFree(c->d_tw_fwd);
    cudaFree(c->d_tw_inv);
    cudaFree(c->d_tw_fwd_wl);
    cudaFree(c->d_tw_inv_wl);
    cudaFree(c->d_cdt);
    cudaFree(c->d_enc_tw);
    cudaFree(c->d_enc_twist);
    cudaFree(c->d_enc_tw_q);
    cudaFree(c->d_enc_twist_q);
    cudaFree(c->d_slot_of);
    cudaFree(c->d_s);
    cudaFree(c->d_pk);
    cudaFree(c->d_pks);
    cudaFree(c->d_ksk);
    for (auto& kv : c->galois) cudaFree(kv.second);
    cudaFree(c->ws);
    cudaFree(c->d_ntt2);
    delete c;
}

// The context's status word: pinned host memory mapped into the device's
// address space, written by a kernel whose bounded wait gave up
static int alloc_status(fhe_ctx* c)
{
    void* h = nullptr;
    cudaError_t e = cudaHostAlloc(&h, sizeof(unsigned int), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *(volatile unsigned int*)h = 0;
        e = cudaHostGetDevicePointer((void**)&c->d_status, h, 0);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h) cudaFreeHost(h);
        return cuda_check(e, "status word");
    }
    c->h_status = (unsigned int*)h;
    return FHE_OK;
}

// Time every NTT schedule on a representative fused step and keep the
// fastest; FHE_NTT_VARIANT fixes both picks, FHE_NTT_VARIANT_KS (with it)
// the key-switching one separately.
static int autotune_ntt(fhe_ctx* c)
{
    const char* env = std::getenv("FHE_NTT_VARIANT");
    if (env && *env) {
        const char* env_ks = std::getenv("FHE_NTT_VARIANT_KS");
        const int v = std::atoi(env), vk = (env_ks && *env_ks) ? std::atoi(env_ks) : v;
        for (int x : {v, vk}) {
            if (x < 0 || x >= kNttVariants) return fail(FHE_EINVAL, "FHE_NTT_VARIANT(_KS) out of range (0..8)");
            if (c->N > kMaxSinglePassN && !ntt_two_pass(x))
                return fail(FHE_EINVAL, "N > 16384 needs a two-pass NTT schedule (2 or 3)");
        }
        c->ntt_variant = v;
        c->ntt_variant_ks = vk;
        c->ntt_forced = true;
        return FHE_OK;
    }
    // Timed workload: a rescale (inverse transform of the last residue, then
    // forward transforms with a fused prologue and epilogue) of 64
    // ciphertexts at the top level, i.e. both directions and the fused I/O the
    // graph kernels use; plain forward transforms when there is nothing to
    // rescale by.
    const uint32_t L = c->L_top;
    const uint32_t rows = c->L_top + 1;
    const uint32_t nct = 64;
    const uint32_t groups = (1216 + rows - 1) / rows;
    const size_t bytes = L >= 2 ? (size_t)nct * 2 * (2 * L) * c->N * 8 : (size_t)groups * rows * c->N * 8;
    u64* buf = nullptr;
    cudaError_t e = cudaMalloc((void**)&buf, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_check(e, "autotune buffer");
    }
    cudaMemset(buf, 0, bytes);
    uint8_t pm[64];
    for (uint32_t r = 0; r < rows; ++r) pm[r] = (uint8_t)r;
    auto work = [&]() {
        if (L >= 2) {
            u64* in = buf;
            u64* out = buf + (size_t)nct * 2 * L * c->N;
            u64* V = out + (size_t)nct * 2 * (L - 1) * c->N;     // fits: 2L residues per ct allocated
            k_rescale(c, in, out, nct, 2, L, nullptr, 0, V, nullptr);
        } else {
            k_ntt_rows(c, buf, groups, rows, pm, true, nullptr);
        }
    };
    const float units = L >= 2 ? (float)(nct * 2 * L) : (float)(groups * rows);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int v = 0; v < kNttVariants; ++v) {
        if (c->N > kMaxSinglePassN && !ntt_two_pass(v)) continue;   // one block per transform needs N <= 16384
        if (ntt_ks_only(v)) continue;                               // key-switching transforms only
        if (v == 8 && !ntt_wl_fits(c->logN)) continue;
        c->ntt_variant = v;
        work();                                                     // warm-up
        float us_best = 1e30f;
        for (int trial = 0; trial < 3 && e == cudaSuccess; ++trial) {
            cudaEventRecord(a, nullptr);
            for (int it = 0; it < 2; ++it) work();
            cudaEventRecord(b, nullptr);
            e = cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            const float us = ms * 1000.f / (2.f * units);
            if (us < us_best) us_best = us;
        }
        if (e != cudaSuccess) break;
        c->ntt_variant_us[v] = us_best;
        if (us_best < best) best = us_best;
    }
    int pick = c->N > kMaxSinglePassN ? 2 : 0;
    for (int v = 0; v < kNttVariants; ++v)
        if (c->ntt_variant_us[v] > 0.f && c->ntt_variant_us[v] == best) { pick = v; break; }
    c->ntt_variant = pick;
    c->ntt_variant_ks = pick;
    cudaFree(buf);
    buf = nullptr;
    // Key-switching digit transforms (key inner product in the epilogue: more
    // registers live) get their own pick, timed on that step alone for
    // min(L_top, 4) digits on zero data (the arithmetic is data-independent),
    // with about 256 MiB of ciphertext data so that, as in real batches, it
    // streams from HBM rather than sitting in L2.  Rings that fit one block
    // per transform only take those schedules here: the two-pass ones add an
    // HBM round trip per digit transform that a small probe would hide.
    if (e == cudaSuccess && c->L_top >= 1) {
        const size_t N = c->N;
        const uint32_t Lk = c->L_top < 4 ? c->L_top : 4;
        const size_t per_ct = (size_t)(3 * Lk + Lk + 2 * (Lk + 1)) * N;
        const uint32_t nk = std::max<uint32_t>(1u, (uint32_t)(((size_t)1 << 25) / per_ct));
        const size_t w_d3 = (size_t)nk * 3 * Lk * N, w_D = (size_t)nk * Lk * N, w_acc = (size_t)nk * 2 * (Lk + 1) * N;
        const size_t w_ksk = (size_t)Lk * 2 * (Lk + 1) * N * 2;
        e = cudaMalloc((void**)&buf, (w_d3 + w_D + w_acc + w_ksk) * 8);
        if (e == cudaSuccess) {
            cudaMemset(buf, 0, (w_d3 + w_D + w_acc + w_ksk) * 8);
            const u64* d3 = buf;
            const u64* D = buf + w_d3;
            u64* acc = buf + w_d3 + w_D;
            const ulonglong2* ksk = (const ulonglong2*)(buf + w_d3 + w_D + w_acc);
            const float kunits = (float)nk * (Lk + 1) * Lk;
            float kbest = 1e30f;
            for (int v = 0; v < kNttVariants && e == cudaSuccess; ++v) {
                if ((c->N > kMaxSinglePassN) != ntt_two_pass(v)) continue;
                if (v == 7 && !modup_cluster_fits(c)) continue;
                if (v == 8 && !ntt_wl_fits(c->logN)) continue;
                c->ntt_variant_ks = v;
                k_modup_mac_step(c, d3, D, ksk, acc, nk, Lk, nullptr);       // warm-up
                float us_best = 1e30f;
                for (int trial = 0; trial < 3 && e == cudaSuccess; ++trial) {
                    cudaEventRecord(a, nullptr);
                    for (int it = 0; it < 2; ++it) k_modup_mac_step(c, d3, D, ksk, acc, nk, Lk, nullptr);
                    cudaEventRecord(b, nullptr);
                    e = cudaEventSynchronize(b);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, a, b);
                    const float us = ms * 1000.f / (2.f * kunits);
                    if (us < us_best) us_best = us;
                }
                c->ntt_variant_ks_us[v] = us_best;
                if (us_best < kbest) kbest = us_best;
            }
            c->ntt_variant_ks = pick;
            for (int v = 0; v < kNttVariants; ++v)
                if (c->ntt_variant_ks_us[v] > 0.f && c->ntt_variant_ks_us[v] == kbest) { c->ntt_variant_ks = v; break; }
            cudaFree(buf);
        } else {
            cudaGetLastError();          // no room for the probe: keep the general pick
            e = cudaSuccess;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_check(e, "autotune");
    return FHE_OK;
}

int fhe_ctx_create(uint32_t N, const uint32_t* bits, uint32_t n_bits, uint32_t log_scale, fhe_ctx** out)
{
    if (!out || !bits) return fail(FHE_EINVAL, "null argument");
    *out = nullptr;
    if (N < 16 || N > 65536 || (N & (N - 1))) return fail(FHE_EUNSUPPORTED, "N must be a power of two in [16, 65536]");
    if (n_bits < 2 || n_bits > 33) return fail(FHE_EINVAL, "need 2..33 coefficient-modulus entries");
    if (log_scale < 1 || log_scale > 60) return fail(FHE_EINVAL, "log_scale out of range");
    std::vector<u64> ch;
    if (!prime_chain(N, bits, n_bits, ch)) return fail(FHE_EINVAL, "bit size out of range [20, 61]");

    fhe_ctx* c = new fhe_ctx();
    c->N = N;
    c->logN = 0;
    while ((1u << c->logN) < N) ++c->logN;
    c->L_top = n_bits - 1;
    c->log_scale = log_scale;
    c->primes = ch;
    c->delta = std::ldexp(1.0, (int)log_scale);
    cudaGetDevice(&c->device);
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        c->sms = 0;
    }

    const uint32_t np = n_bits;
    c->pc.resize(np);
    std::vector<ulonglong2> twf((size_t)np * N), twi((size_t)np * N);
    for (uint32_t r = 0; r < np; ++r) {
        const u64 q = ch[r];
        PrimeC& P = c->pc[r];
        P.q = q;
        P.q2 = 2 * q;
        P.mu = (u64)(((u128)1 << 64) / q);
        P.r64 = (u64)(((u128)1 << 64) % q);
        P.r64s = shoup(P.r64, q);
        P.ninv = hinv(N, q);
        P.ninvs = shoup(P.ninv, q);
        P.half = (q - 1) / 2;
        P.ub = (u64)((((u128)1 << 64) / q) * q);
        for (int k = 0; k < 4; ++k) {
            P.p21[k] = hpow(2, 21ull * (k + 1), q);
            P.p21s[k] = shoup(P.p21[k], q);
        }
        {
            int b = 0;
            while (b < 64 && (q >> b)) ++b;                  // bit length of q (q < 2^62)
            P.bsh = (u64)(b - 1);
            P.bmu = (u64)((((u128)1 << (2 * b)) / q) << (63 - b));
        }
        const u64 psi = primitive_root_2n(q, N);
        const u64 psi_inv = hinv(psi, q);
        for (uint32_t i = 0; i < N; ++i) {
            const uint32_t br = bitrev(i, (int)c->logN);
            const u64 w = hpow(psi, br, q), wi = hpow(psi_inv, br, q);
            twf[(size_t)r * N + i] = make_ulonglong2(w, shoup(w, q));
            twi[(size_t)r * N + i] = make_ulonglong2(wi, shoup(wi, q));
        }
    }
    // warp-local layouts: the stages whose twiddles vary per lane (forward:
    // the last five, 2^t entries per lane at stage log2 N - 5 + t; inverse:
    // the first five, 2^(4-s) per lane at stage s) transposed by wl_perm
    std::vector<ulonglong2> twf_wl, twi_wl;
    if (ntt_wl_fits(c->logN)) {
        twf_wl = twf;
        twi_wl = twi;
        const int lg = (int)c->logN;
        for (uint32_t r = 0; r < np; ++r) {
            const size_t o = (size_t)r * N;
            for (int t = 0; t < 5; ++t) {
                const uint32_t base = 1u << (lg - 5 + t);
                for (uint32_t k = 0; k < base; ++k) twf_wl[o + base + wl_perm(k, t)] = twf[o + base + k];
            }
            for (int st = 0; st < 5; ++st) {
                const uint32_t base = N >> (st + 1);
                for (uint32_t k = 0; k < base; ++k) twi_wl[o + base + wl_perm(k, 4 - st)] = twi[o + base + k];
            }
        }
    }
    std::vector<u64> cdt = gauss_cdt();
    // encoder tables: zeta^{-4k} (k < N/4), zeta^{-k} (k < N/2), slot positions
    std::vector<double4> etw(N / 4), etwist(N / 2);
    std::vector<ulonglong2> etw_q(N / 2), etwist_q(N);
    auto q126 = [](const dd& v) {
        u64 lo, hi;
        dd_to_q126(v, &lo, &hi);
        return make_ulonglong2(lo, hi);
    };
    for (uint32_t k = 0; k < N / 4; ++k) {
        cdd z = zeta_pow_dd(-4 * (int64_t)k, N);
        etw[k] = make_double4(z.re.hi, z.re.lo, z.im.hi, z.im.lo);
        etw_q[2 * k] = q126(z.re);
        etw_q[2 * k + 1] = q126(z.im);
    }
    for (uint32_t k = 0; k < N / 2; ++k) {
        cdd z = zeta_pow_dd(-(int64_t)k, N);
        etwist[k] = make_double4(z.re.hi, z.re.lo, z.im.hi, z.im.lo);
        etwist_q[2 * k] = q126(z.re);
        etwist_q[2 * k + 1] = q126(z.im);
    }
    std::vector<uint32_t> slot_of(N / 2);
    u64 e = 1;
    for (uint32_t j = 0; j < N / 2; ++j) {
        slot_of[(e - 1) / 4] = j;
        e = (e * 5) % (2ull * N);
    }

    int rc = FHE_OK;
    auto up = [&](void** dst, const void* src, size_t bytes) {
        if (rc != FHE_OK) return;
        cudaError_t err = cudaMalloc(dst, bytes);
        if (err == cudaSuccess) err = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
        if (err != cudaSuccess) {
            cudaGetLastError();
            rc = cuda_check(err, "fhe_ctx_create upload");
        }
    };
    up((void**)&c->d_pc, c->pc.data(), np * sizeof(PrimeC));
    up((void**)&c->d_tw_fwd, twf.data(), twf.size() * sizeof(ulonglong2));
    up((void**)&c->d_tw_inv, twi.data(), twi.size() * sizeof(ulonglong2));
    if (!twf_wl.empty()) {
        up((void**)&c->d_tw_fwd_wl, twf_wl.data(), twf_wl.size() * sizeof(ulonglong2));
        up((void**)&c->d_tw_inv_wl, twi_wl.data(), twi_wl.size() * sizeof(ulonglong2));
    }
    up((void**)&c->d_cdt, cdt.data(), cdt.size() * sizeof(u64));
    up((void**)&c->d_enc_tw, etw.data(), etw.size() * sizeof(double4));
    up((void**)&c->d_enc_twist, etwist.data(), etwist.size() * sizeof(double4));
    up((void**)&c->d_enc_tw_q, etw_q.data(), etw_q.size() * sizeof(ulonglong2));
    up((void**)&c->d_enc_twist_q, etwist_q.data(), etwist_q.size() * sizeof(ulonglong2));
    up((void**)&c->d_slot_of, slot_of.data(), slot_of.size() * sizeof(uint32_t));
    if (rc == FHE_OK) rc = alloc_status(c);
    if (rc == FHE_OK) {
        // two-pass NTT intermediate: 128 MiB (or 64 transforms for small rings)
        c->ntt2_words = std::max<size_t>((size_t)1 << 24, (size_t)64 * N);
        cudaError_t err = cudaMalloc((void**)&c->d_ntt2, c->ntt2_words * 8);
        if (err != cudaSuccess) {
            cudaGetLastError();
            rc = cuda_check(err, "two-pass NTT scratch");
        }
    }
    if (rc != FHE_OK) {
        free_ctx(c);
        return rc;
    }
    c->key_bytes = np * sizeof(PrimeC) + 2 * (twf.size() + twf_wl.size()) * sizeof(ulonglong2) + cdt.size() * 8 +
                   (etw.size() + etwist.size()) * sizeof(double4) +
                   (etw_q.size() + etwist_q.size()) * sizeof(ulonglong2) + slot_of.size() * 4;
    rc = autotune_ntt(c);
    if (rc != FHE_OK) {
        free_ctx(c);
        return rc;
    }
    *out = c;
    return FHE_OK;
}

int fhe_ctx_fork(fhe_ctx* parent, fhe_ctx** out)
{
    CHECK_CTX(parent);
    if (!out) return fail(FHE_EINVAL, "null output");
    *out = nullptr;
    if (parent->parent) parent = parent->parent;
    fhe_ctx* c = new fhe_ctx();
    c->N = parent->N;
    c->logN = parent->logN;
    c->L_top = parent->L_top;
    c->log_scale = parent->log_scale;
    c->primes = parent->primes;
    c->pc = parent->pc;
    c->delta = parent->delta;
    c->device = parent->device;
    c->ntt_variant = parent->ntt_variant;
    c->ntt_variant_ks = parent->ntt_variant_ks;
    c->ntt_forced = parent->ntt_forced;
    c->sms = parent->sms;
    for (int v = 0; v < 16; ++v) {
        c->ntt_variant_us[v] = parent->ntt_variant_us[v];
        c->ntt_variant_ks_us[v] = parent->ntt_variant_ks_us[v];
    }
    c->d_pc = parent->d_pc;
    c->d_tw_fwd = parent->d_tw_fwd;
    c->d_tw_inv = parent->d_tw_inv;
    c->d_tw_fwd_wl = parent->d_tw_fwd_wl;
    c->d_tw_inv_wl = parent->d_tw_inv_wl;
    c->d_cdt = parent->d_cdt;
    c->d_enc_tw = parent->d_enc_tw;
    c->d_enc_twist = parent->d_enc_twist;
    c->d_enc_tw_q = parent->d_enc_tw_q;
    c->d_enc_twist_q = parent->d_enc_twist_q;
    c->d_slot_of = parent->d_slot_of;
    c->has_keys = parent->has_keys;
    c->seed = parent->seed;
    c->d_s = parent->d_s;
    c->d_pk = parent->d_pk;
    c->d_pks = parent->d_pks;
    c->d_ksk = parent->d_ksk;
    c->parent = parent;
    c->ntt2_words = parent->ntt2_words;
    cudaError_t e = cudaMalloc((void**)&c->d_ntt2, c->ntt2_words * 8);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return cuda_check(e, "fork scratch");
    }
    const int rc = alloc_status(c);
    if (rc != FHE_OK) {
        free_ctx(c);
        return rc;
    }
    *out = c;
    return FHE_OK;
}

int fhe_ctx_destroy(fhe_ctx* c)
{
    if (!c) return FHE_OK;
    cudaDeviceSynchronize();
    free_ctx(c);
    return FHE_OK;
}

int fhe_ctx_query(const fhe_ctx* c, fhe_ctx_info* out)
{
    CHECK_CTX(c);
    if (!out) return fail(FHE_EINVAL, "null output");
    std::memset(out, 0, sizeof(*out));
    out->N = c->N;
    out->slots = c->N / 2;
    out->L_top = c->L_top;
    out->log_scale = c->log_scale;
    for (size_t i = 0; i < c->primes.size() && i < 64; ++i) out->primes[i] = c->primes[i];
    out->key_bytes = c->key_bytes;
    out->ntt_variant = (uint32_t)c->ntt_variant;
    out->ntt_variant_ks = (uint32_t)c->ntt_variant_ks;
    out->workspace_bytes = c->ws_bytes + c->bb_bytes;
    for (int v = 0; v < kNttVariants && v < 16; ++v) {
        out->ntt_variant_us[v] = c->ntt_variant_us[v];
        out->ntt_variant_ks_us[v] = c->ntt_variant_ks_us[v];
    }
    return FHE_OK;
}

int fhe_keygen(fhe_ctx* c, uint64_t seed, void* stream)
{
    CHECK_CTX(c);
    if (c->parent) return fail(FHE_EINVAL, "keygen on a fork: generate keys on the parent context");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = c->N, Lt = c->L_top;
    if (!c->d_s) {
        size_t bs = (Lt + 1) * N * 8, bp = 2 * Lt * N * 8, bk = Lt * 2 * (Lt + 1) * N * 16;
        cudaError_t e = cudaMalloc((void**)&c->d_s, bs);
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_pk, bp);
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_pks, bp);
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_ksk, bk);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_check(e, "key allocation");
        }
        c->key_bytes += bs + 2 * bp + bk;
    }
    c->seed = seed;
    k_keygen(c, st);
    CUDA_LAST("keygen launch");
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(e, "keygen");
    c->has_keys = true;
    return FHE_OK;
}

int fhe_export_secret(fhe_ctx* c, uint64_t* d_out, void* stream)
{
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (!d_out) return fail(FHE_EINVAL, "null output");
    return cuda_check(cudaMemcpyAsync(d_out, c->d_s, (size_t)(c->L_top + 1) * c->N * 8, cudaMemcpyDeviceToDevice,
                                      (cudaStream_t)stream),
                      "export secret");
}

// ---------------------------------------------------------------- encode etc.
int fhe_encode(fhe_ctx* c, const double* d_slots, uint32_t n_ct, uint32_t level, double scale, uint64_t* d_pt,
               void* stream)
{
    CHECK_CTX(c);
    if (n_ct == 0) return FHE_OK;
    if (!d_slots || !d_pt) return fail(FHE_EINVAL, "null buffer");
    if (level < 1 || level > c->L_top) return fail(FHE_ELEVEL, "level out of range");
    if (!(scale > 0.0) || !std::isfinite(scale)) return fail(FHE_EINVAL, "bad scale");
    Arena ar;
    int rc = ws_reserve(c, encode_scratch_bytes(c, n_ct), &ar);
    if (rc) return rc;
    k_encode(c, d_slots, n_ct, level, scale, (u64*)d_pt, ar.take(encode_scratch_bytes(c, n_ct)), (cudaStream_t)stream);
    CUDA_LAST("encode launch");
    return FHE_OK;
}

int fhe_encrypt(fhe_ctx* c, const uint64_t* d_pt, uint32_t n_ct, uint64_t first_ct_id, uint64_t* d_ct, void* stream)
{
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (n_ct == 0) return FHE_OK;
    if (!d_pt || !d_ct) return fail(FHE_EINVAL, "null buffer");
    Arena ar;
    const size_t need = encrypt_scratch_bytes(c, n_ct);
    int rc = ws_reserve(c, need, &ar);
    if (rc) return rc;
    k_encrypt(c, (const u64*)d_pt, n_ct, first_ct_id, (u64*)d_ct, ar.take(need), (cudaStream_t)stream);
    CUDA_LAST("encrypt launch");
    return FHE_OK;
}

int fhe_encode_encrypt(fhe_ctx* c, const double* d_slots, uint32_t n_ct, double scale, uint64_t first_ct_id,
                       uint64_t* d_ct, void* stream)
{
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (n_ct == 0) return FHE_OK;
    if (!d_slots || !d_ct) return fail(FHE_EINVAL, "null buffer");
    if (!(scale > 0.0) || !std::isfinite(scale)) return fail(FHE_EINVAL, "bad scale");
    Arena ar;
    const size_t need = encode_encrypt_scratch_bytes(c, n_ct);
    int rc = ws_reserve(c, need, &ar);
    if (rc) return rc;
    k_encode_encrypt(c, d_slots, n_ct, scale, first_ct_id, (u64*)d_ct, ar.take(need), (cudaStream_t)stream);
    CUDA_LAST("encode_encrypt launch");
    return FHE_OK;
}

int fhe_decrypt(fhe_ctx* c, const uint64_t* d_ct, uint32_t n_ct, uint32_t level, int64_t* d_m, void* stream)
{
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (n_ct == 0) return FHE_OK;
    if (!d_ct || !d_m) return fail(FHE_EINVAL, "null buffer");
    if (level < 1 || level > c->L_top) return fail(FHE_ELEVEL, "level out of range");
    k_decrypt(c, (const u64*)d_ct, n_ct, level, (i64*)d_m, (cudaStream_t)stream);
    CUDA_LAST("decrypt launch");
    return FHE_OK;
}

int fhe_decode(fhe_ctx* c, const int64_t* d_m, uint32_t n_ct, double scale, double* d_slots, void* stream)
{
    CHECK_CTX(c);
    if (n_ct == 0) return FHE_OK;
    if (!d_m || !d_slots) return fail(FHE_EINVAL, "null buffer");
    if (!(scale > 0.0) || !std::isfinite(scale)) return fail(FHE_EINVAL, "bad scale");
    k_decode(c, (const i64*)d_m, n_ct, scale, d_slots, (cudaStream_t)stream);
    CUDA_LAST("decode launch");
    return FHE_OK;
}

int fhe_ntt(fhe_ctx* c, uint64_t* d_poly, uint32_t n_poly, uint32_t rows, int forward, void* stream)
{
    CHECK_CTX(c);
    if (n_poly == 0) return FHE_OK;
    if (!d_poly) return fail(FHE_EINVAL, "null buffer");
    if (rows < 1 || rows > c->L_top + 1) return fail(FHE_EINVAL, "rows out of range");
    uint8_t pm[64];
    for (uint32_t r = 0; r < rows; ++r) pm[r] = (uint8_t)r;
    k_ntt_rows(c, (u64*)d_poly, n_poly, rows, pm, forward != 0, (cudaStream_t)stream);
    CUDA_LAST("ntt launch");
    return FHE_OK;
}

int fhe_ct_convert(fhe_ctx* c, const uint64_t* d_in, uint32_t n_ct, uint32_t level, int to_coeff, uint64_t* d_out,
                   void* stream)
{
    CHECK_CTX(c);
    if (n_ct == 0) return FHE_OK;
    if (!d_in || !d_out) return fail(FHE_EINVAL, "null buffer");
    if (level < 1 || level > c->L_top) return fail(FHE_ELEVEL, "level out of range");
    k_ct_to_coeff(c, (const u64*)d_in, (u64*)d_out, n_ct, 2, level, to_coeff != 0, (cudaStream_t)stream);
    CUDA_LAST("convert launch");
    return FHE_OK;
}

// ---------------------------------------------------------------- ops
#define CHECK_LEVEL(c, L, lo)                                                  \
    do {                                                                       \
        if ((L) < (lo) || (L) > (c)->L_top) return fail(FHE_ELEVEL, "level out of range"); \
    } while (0)

int fhe_add(fhe_ctx* c, const uint64_t* a, const uint64_t* b, uint32_t n_ct, uint32_t level, uint64_t* out,
            void* stream)
{
    CHECK_CTX(c);
    CHECK_LEVEL(c, level, 1);
    if (n_ct == 0) return FHE_OK;
    if (!a || !b || !out) return fail(FHE_EINVAL, "null buffer");
    k_add(c, (const u64*)a, (const u64*)b, (u64*)out, n_ct, 2, level, (cudaStream_t)stream);
    CUDA_LAST("add launch");
    return FHE_OK;
}

int fhe_tensor(fhe_ctx* c, const uint64_t* a, const uint64_t* b, uint32_t n_ct, uint32_t level, uint64_t* out,
               void* stream)
{
    CHECK_CTX(c);
    CHECK_LEVEL(c, level, 1);
    if (n_ct == 0) return FHE_OK;
    if (!a || !b || !out) return fail(FHE_EINVAL, "null buffer");
    k_tensor(c, (const u64*)a, (const u64*)b, (u64*)out, n_ct, level, (cudaStream_t)stream);
    CUDA_LAST("tensor launch");
    return FHE_OK;
}

int fhe_relinearise(fhe_ctx* c, const uint64_t* d3, uint32_t n_ct, uint32_t level, uint64_t* out, void* stream)
{
    CHECK_CTX(c);
    CHECK_KEYS(c);
    CHECK_LEVEL(c, level, 1);
    if (n_ct == 0) return FHE_OK;
    if (!d3 || !out) return fail(FHE_EINVAL, "null buffer");
    Arena ar;
    size_t need = relin_scratch_bytes(c, n_ct, level);
    int rc = ws_reserve(c, need, &ar);
    if (rc) return rc;
    k_relin(c, (const u64*)d3, (u64*)out, n_ct, level, ar.take(need), (cudaStream_t)stream);
    CUDA_LAST("relinearise launch");
    return FHE_OK;
}

int fhe_galois_keygen(fhe_ctx* c, const int32_t* steps, uint32_t n_steps, void* stream)
{
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (c->parent) return fail(FHE_EINVAL, "generate rotation keys on the parent context");
    if (n_steps && !steps) return fail(FHE_EINVAL, "null steps");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int64_t> v(steps, steps + n_steps);
    int rc = galois_keys_for(c, v, st);
    if (rc) return rc;
    CUDA_LAST("rotation keygen launch");
    return cuda_check(cudaStreamSynchronize(st), "rotation keygen");
}

int fhe_gather_slots(const double* d_src, const int64_t* d_index, uint32_t rows, uint32_t cols, double* d_dst,
                     void* stream)
{
    if ((size_t)rows * cols == 0) return FHE_OK;
    if (!d_src || !d_index || !d_dst) return fail(FHE_EINVAL, "null buffer");
    k_gather_slots(d_src, d_index, (size_t)rows * cols, d_dst, (cudaStream_t)stream);
    CUDA_LAST("gather launch");
    return FHE_OK;
}

int fhe_rotate(fhe_ctx* c, const uint64_t* d_ct, uint32_t n_ct, uint32_t level, int32_t step, uint64_t* d_out,
               void* stream)
{
    CHECK_CTX(c);
    CHECK_KEYS(c);
    CHECK_LEVEL(c, level, 1);
    if (n_ct == 0) return FHE_OK;
    if (!d_ct || !d_out) return fail(FHE_EINVAL, "null buffer");
    const u64 k = galois_element_of(c, step);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t w = (size_t)n_ct * 2 * level * c->N * 8;
    if (k == 1) {
        if (d_out == d_ct) return FHE_OK;
        return cuda_check(cudaMemcpyAsync(d_out, d_ct, w, cudaMemcpyDeviceToDevice, st), "rotate copy");
    }
    const fhe_ctx* root = c->parent ? c->parent : c;
    auto it = root->galois.find(k);
    if (it == root->galois.end()) return fail(FHE_ENOKEY, "no rotation key for this step (fhe_galois_keygen)");
    Arena ar;
    const size_t d3b = (size_t)n_ct * 3 * level * c->N * 8, rs = relin_scratch_bytes(c, n_ct, level);
    int rc = ws_reserve(c, arena_need({d3b, rs}), &ar);
    if (rc) return rc;
    u64* d3 = (u64*)ar.take(d3b);
    k_automorph(c, (const u64*)d_ct, d3, n_ct, level, k, st);
    k_relin(c, d3, (u64*)d_out, n_ct, level, ar.take(rs), st, it->second);
    CUDA_LAST("rotate launch");
    return FHE_OK;
}

int fhe_rescale(fhe_ctx* c, const uint64_t* in, uint32_t n_ct, uint32_t comps, uint32_t level, uint64_t* out,
                void* stream)
{
    CHECK_CTX(c);
    CHECK_LEVEL(c, level, 2);
    if (n_ct == 0) return FHE_OK;
    if (!in || !out) return fail(FHE_EINVAL, "null buffer");
    if (comps < 1 || comps > 3) return fail(FHE_EINVAL, "comps must be 1..3");
    Arena ar;
    size_t need = rescale_scratch_bytes(c, n_ct, comps);
    int rc = ws_reserve(c, need, &ar);
    if (rc) return rc;
    k_rescale(c, (const u64*)in, (u64*)out, n_ct, comps, level, nullptr, 0, ar.take(need), (cudaStream_t)stream);
    CUDA_LAST("rescale launch");
    return FHE_OK;
}

int fhe_mul_relin_rescale(fhe_ctx* c, const uint64_t* a, const uint64_t* b, uint32_t n_ct, uint32_t level,
                          uint64_t* out, void* stream)
{
    CHECK_CTX(c);
    CHECK_KEYS(c);
    CHECK_LEVEL(c, level, 2);
    if (n_ct == 0) return FHE_OK;
    if (!a || !b || !out) return fail(FHE_EINVAL, "null buffer");
    const size_t N = c->N;
    const size_t wa = (size_t)n_ct * 2 * level * N, wo = (size_t)n_ct * 2 * (level - 1) * N;
    auto overlaps = [&](const uint64_t* x) { return x < out + wo && out < x + wa; };
    // the factors are read until the last step, which writes d_out: when
    // d_out overlaps them, the tensor is formed first
    const bool fused = !overlaps(a) && !overlaps(b);
    const size_t b3 = fused ? 0 : (size_t)n_ct * 3 * level * N * 8, br = relin_rescale_scratch_bytes(c, n_ct, level);
    Arena ar;
    int rc = ws_reserve(c, arena_need({b3, br}), &ar);
    if (rc) return rc;
    u64* t3 = fused ? nullptr : (u64*)ar.take(b3);
    void* sr = ar.take(br);
    cudaStream_t st = (cudaStream_t)stream;
    if (fused) {
        k_mul_relin_rescale(c, (const u64*)a, (const u64*)b, (u64*)out, n_ct, level, sr, st);
    } else {
        k_tensor(c, (const u64*)a, (const u64*)b, t3, n_ct, level, st);
        k_relin_rescale(c, t3, (u64*)out, n_ct, level, sr, st);
    }
    CUDA_LAST("mul_relin_rescale launch");
    return FHE_OK;
}

int fhe_mul_relin_rescale_levels(fhe_ctx* c, const fhe_level_batch* batches, uint32_t n_batches, void* stream)
{
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (n_batches == 0) return FHE_OK;
    if (!batches) return fail(FHE_EINVAL, "null batch table");
    if (c->N > kMaxSinglePassN) return fail(FHE_EUNSUPPORTED, "grouped steps need N <= 16384");
    for (uint32_t k = 0; k < n_batches; ++k) {
        const fhe_level_batch& b = batches[k];
        if (b.level < 2 || b.level > c->L_top) return fail(FHE_ELEVEL, "batch level out of range");
        if (b.n_ct && (!b.d_a || !b.d_b || !b.d_out)) return fail(FHE_EINVAL, "null batch buffer");
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (uint32_t k0 = 0; k0 < n_batches; k0 += kMaxLevelBatches) {
        LevelBatch g[kMaxLevelBatches];
        int ng = 0;
        for (uint32_t k = k0; k < n_batches && k < k0 + kMaxLevelBatches; ++k) {
            if (batches[k].n_ct == 0) continue;
            g[ng++] = LevelBatch{(const u64*)batches[k].d_a, (const u64*)batches[k].d_b, (u64*)batches[k].d_out,
                                 batches[k].n_ct, batches[k].level};
        }
        if (ng == 0) continue;
        // FHE_PERSISTENT=0 runs the six-launch form instead (for comparisons)
        const char* env = std::getenv("FHE_PERSISTENT");
        const bool persistent = !(env && env[0] == '0');
        const size_t need = persistent ? persist_scratch_bytes(c, g, ng) : level_groups_scratch_bytes(c, g, ng);
        Arena ar;
        int rc = ws_reserve(c, need, &ar);
        if (rc) return rc;
        if (persistent) {
            rc = k_mul_relin_rescale_persistent(c, g, ng, ar.take(need), st);
            if (rc) return rc;
        } else {
            k_mul_relin_rescale_groups(c, g, ng, ar.take(need), st);
        }
        CUDA_LAST("mul_relin_rescale_levels launch");
    }
    return FHE_OK;
}

static int upload_const_residues(fhe_ctx* c, const int64_t* h, uint32_t n_ct, uint32_t level, Arena* ar, u64** dres,
                                 cudaStream_t st)
{
    std::vector<u64> res((size_t)n_ct * level);
    for (uint32_t k = 0; k < n_ct; ++k)
        for (uint32_t r = 0; r < level; ++r) res[(size_t)k * level + r] = mod_signed(h[k], c->primes[r]);
    *dres = (u64*)ar->take(res.size() * 8);
    return cuda_check(cudaMemcpyAsync(*dres, res.data(), res.size() * 8, cudaMemcpyHostToDevice, st), "const upload");
}

int fhe_mul_const(fhe_ctx* c, const uint64_t* in, const int64_t* h_c, uint32_t n_ct, uint32_t level, uint64_t* out,
                  void* stream)
{
    CHECK_CTX(c);
    CHECK_LEVEL(c, level, 1);
    if (n_ct == 0) return FHE_OK;
    if (!in || !out || !h_c) return fail(FHE_EINVAL, "null buffer");
    Arena ar;
    int rc = ws_reserve(c, (size_t)n_ct * level * 8 + 256, &ar);
    if (rc) return rc;
    u64* dres;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = upload_const_residues(c, h_c, n_ct, level, &ar, &dres, st))) return rc;
    k_mul_const(c, (const u64*)in, (u64*)out, n_ct, 2, level, level, dres, level, st);
    CUDA_LAST("mul_const launch");
    return cuda_check(cudaStreamSynchronize(st), "mul_const");
}

int fhe_add_const(fhe_ctx* c, uint64_t* ct, const int64_t* h_c, uint32_t n_ct, uint32_t level, void* stream)
{
    CHECK_CTX(c);
    CHECK_LEVEL(c, level, 1);
    if (n_ct == 0) return FHE_OK;
    if (!ct || !h_c) return fail(FHE_EINVAL, "null buffer");
    Arena ar;
    int rc = ws_reserve(c, (size_t)n_ct * level * 8 + 256, &ar);
    if (rc) return rc;
    u64* dres;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = upload_const_residues(c, h_c, n_ct, level, &ar, &dres, st))) return rc;
    k_add_const(c, (u64*)ct, n_ct, level, dres, level, st);
    CUDA_LAST("add_const launch");
    return cuda_check(cudaStreamSynchronize(st), "add_const");
}

// ---------------------------------------------------------------- measurement
static const char* kFamilies =
    "ntt,rescale_intt,rescale_ntt,keyswitch_intt,keyswitch_modup_mac,keyswitch_acc_intt,keyswitch_moddown,"
    "keyswitch_rescale_intt,keyswitch_rescale_ntt,"
    "keygen,encrypt,decrypt,encode_ntt,encode_fft,decode_fft,mac,mac_tc,tensor,elementwise,persistent";

const char* fhe_profile_families(void) { return kFamilies; }

int fhe_profile_begin(fhe_ctx* c, const char* family, uint32_t max_launches)
{
    CHECK_CTX(c);
    if (!family || !*family) return fail(FHE_EINVAL, "empty family");
    std::string f(family);
    std::string all = std::string(",") + kFamilies + ",";
    if (all.find("," + f + ",") == std::string::npos) return fail(FHE_EINVAL, "unknown kernel family " + f);
    if (max_launches == 0) max_launches = 1;
    while (c->prof_ev.size() < 2 * (size_t)max_launches) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return cuda_check(err, "cudaEventCreate");
        c->prof_ev.push_back(e);
    }
    c->prof_family = f;
    c->prof_used = 0;
    c->prof_launches = 0;
    return FHE_OK;
}

int fhe_profile_end(fhe_ctx* c, double* total_ms, uint64_t* launches, uint64_t* timed)
{
    CHECK_CTX(c);
    double tot = 0.0;
    for (size_t i = 0; i + 1 < c->prof_used; i += 2) {
        cudaError_t e = cudaEventSynchronize(c->prof_ev[i + 1]);
        if (e != cudaSuccess) return cuda_check(e, "profile event");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->prof_ev[i], c->prof_ev[i + 1]);
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = c->prof_launches;
    if (timed) *timed = c->prof_used / 2;
    c->prof_family.clear();
    c->prof_used = 0;
    c->prof_launches = 0;
    return FHE_OK;
}

int fhe_launch_count(uint64_t* out)
{
    if (!out) return fail(FHE_EINVAL, "null output");
    *out = launch_count();
    return FHE_OK;
}

int fhe_ctx_sync(fhe_ctx* c, void* stream)
{
    CHECK_CTX(c);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_check(e, "fhe_ctx_sync");
    return status_take(c);
}

int fhe_inject_fault(fhe_ctx* c, uint32_t kind)
{
    CHECK_CTX(c);
    if (kind != FHE_INJECT_MAC_TC_WITHHOLD && kind != FHE_INJECT_PERSIST_STALL)
        return fail(FHE_EINVAL, "unknown fault kind");
    c->inject = (int)kind;
    return FHE_OK;
}

int fhe_device_faults(uint32_t* out)
{
    if (!out) return fail(FHE_EINVAL, "null output");
    *out = fhe::mac_tc_fault_take();
    if (*out == 0xFFFFFFFFu) return fail(FHE_ECUDA, "reading the device fault flags failed");
    return FHE_OK;
}

}  // extern "C"
