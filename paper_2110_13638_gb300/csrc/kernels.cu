// kernels.cu -- sm_103a kernels of the RNS-CKKS path.
//
// Every transform-bearing step is one launch of k_ntt_op (fhe_device.cuh)
// with a step-specific Op whose load() is the fused prologue (sampling,
// base conversion, pointwise products) and whose store() is the fused
// epilogue (key products, ModDown / rescale combination, encryption sums).
// The remaining kernels are element-wise (coalesced, grid-stride), the
// gather multiply-accumulate of dense / convolution layers, and the
// double-double / FP64 canonical-embedding FFTs of encode / decode.
#include <algorithm>
#include <atomic>
#include <cstdio>

#include "ctx.h"
#include "host_math.h"

namespace fhe {

static constexpr u64 kGamma = 0x9E3779B97F4A7C15ull;

// ---------------------------------------------------------------- PRNG
// SplitMix64 (Steele, Lea, Flood 2014): output i of the generator started in
// state s is mix(s + (i + 1) * gamma).  Draw index = coef | residue << 16 | retry << 24.
__host__ __device__ __forceinline__ u64 mix64(u64 z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ u64 sm_out(u64 s, u64 i) { return mix64(s + (i + 1) * kGamma); }

uint64_t stream_key(uint64_t seed, uint64_t domain, uint64_t object)
{
    return sm_out(sm_out(seed, domain), object);
}

__device__ __forceinline__ i64 draw_ternary(u64 s0, int j)
{
    const u64 bound = 0xFFFFFFFFFFFFFFFFull;     // 3 * floor(2^64 / 3) = 2^64 - 1
    for (u64 t = 0;; ++t) {
        u64 u = sm_out(s0, (u64)j | (t << 24));
        if (u < bound) return (i64)(u % 3ull) - 1;
    }
}

__device__ __forceinline__ i64 draw_gauss(u64 s0, int j, const u64* __restrict__ cdt)
{
    u64 u = sm_out(s0, (u64)j);
    i64 e = -19;
#pragma unroll
    for (int i = 0; i < 38; ++i) e += (u >= __ldg(&cdt[i])) ? 1 : 0;
    return e;
}

__device__ __forceinline__ u64 draw_uniform(u64 s0, int j, int r, const PrimeC& P)
{
    for (u64 t = 0;; ++t) {
        u64 u = sm_out(s0, (u64)j | ((u64)r << 16) | (t << 24));
        if (u < P.ub) return reduce64(u, P);
    }
}

// ---------------------------------------------------------------- launch
static std::atomic<uint64_t> g_launches{0};

uint64_t launch_count() { return g_launches.load(); }

LaunchScope::LaunchScope(const fhe_ctx* ctx, const char* family, cudaStream_t s) : c(ctx), st(s)
{
    g_launches.fetch_add(1);
    if (!c->prof_family.empty() && c->prof_family == family) {
        c->prof_launches += 1;
        if (c->prof_used + 2 <= c->prof_ev.size()) {
            idx = (long)c->prof_used;
            c->prof_used += 2;
            cudaEventRecord(c->prof_ev[idx], st);
        }
    }
}

LaunchScope::~LaunchScope()
{
    if (idx >= 0) cudaEventRecord(c->prof_ev[idx + 1], st);
}

// NTT schedule variants (radix of the register passes, threads per block);
// the context's autotuner picks one per ring degree.
template <bool INV, int LOGR, int MAXT, class Op>
static void launch_ntt_v(const fhe_ctx* c, const Op& op, int count, cudaStream_t st)
{
    const int N = (int)c->N;
    int thr = N >> LOGR;
    thr = thr < 32 ? 32 : (thr > MAXT ? MAXT : thr);
    const size_t smem = (size_t)ntt_smem_words(N) * sizeof(u64);
    auto fn = k_ntt_op<INV, LOGR, MAXT, Op>;
    static size_t configured = 0;        // per instantiation
    if (configured < smem) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = smem;
    }
    LaunchScope ls(c, Op::family(), st);
    fn<<<count, thr, smem, st>>>(op, c->tabs());
}

// Several batches of one transform step, each with its own level, in ONE
// launch: unit p is located in the group table by prefix sums.
constexpr int kMaxGroups = 8;

template <class Op>
struct MultiOp {
    static const char* family() { return Op::family(); }
    typedef typename Op::Pre Pre;
    Op ops[kMaxGroups];
    int pre_[kMaxGroups + 1];
    int ng;
    __host__ __device__ int count() const { return pre_[ng]; }
    __host__ __device__ int locate(int p, int& q) const
    {
        int g = 0;
        while (g + 1 < ng && p >= pre_[g + 1]) ++g;
        q = p - pre_[g];
        return g;
    }
    __host__ __device__ int nsub(int p) const
    {
        int q;
        const int g = locate(p, q);
        return ops[g].nsub(q);
    }
    __device__ int prime(int p, int u) const
    {
        int q;
        const int g = locate(p, q);
        return ops[g].prime(q, u);
    }
    __device__ bool direct(int p, int u) const
    {
        int q;
        const int g = locate(p, q);
        return ops[g].direct(q, u);
    }
    __device__ u64 load(int p, int u, int j, const PrimeC& P) const
    {
        int q;
        const int g = locate(p, q);
        return ops[g].load(q, u, j, P);
    }
    __device__ Pre pre(int p, int u, int j) const
    {
        int q;
        const int g = locate(p, q);
        return ops[g].pre(q, u, j);
    }
    __device__ void store(int p, int u, int j, u64 v, const Pre& pr, const PrimeC& P) const
    {
        int q;
        const int g = locate(p, q);
        ops[g].store(q, u, j, v, pr, P);
    }
};

template <class Op> struct uniform_subs { static constexpr bool value = true; };
template <class Op> struct uniform_subs<MultiOp<Op>> { static constexpr bool value = false; };

// two-pass schedule: column / row tiles, intermediate in the context's
// scratch, units processed in chunks that fit it
template <bool INV, int LOGR, class Op>
static void launch_ntt_2pass(const fhe_ctx* c, const Op& op, int count, cudaStream_t st)
{
    Split2 sp;
    sp.k1 = (int)c->logN / 2;
    sp.k2 = (int)c->logN - sp.k1;
    const int N1 = 1 << sp.k1, N2 = 1 << sp.k2, N = (int)c->N;
    sp.cs = N2 < kTile2 ? N2 : kTile2;
    sp.rs = N1 < kTile2 ? N1 : kTile2;
    const int ns = op.nsub(0);
    const size_t words = (size_t)(N1 * sp.cs > sp.rs * ntt_smem_words(N2) ? N1 * sp.cs : sp.rs * ntt_smem_words(N2));
    const size_t smem = words * sizeof(u64);
    int chunk = (int)(c->ntt2_words / ((size_t)ns * N));
    if (chunk < 1) chunk = 1;
    const int t1 = INV ? N1 / sp.rs : N2 / sp.cs;      // tiles of the first pass
    const int t2 = INV ? N2 / sp.cs : N1 / sp.rs;      // tiles of the second pass
    for (int p0 = 0; p0 < count; p0 += chunk) {
        sp.p0 = p0;
        sp.nunits = count - p0 < chunk ? count - p0 : chunk;
        {
            LaunchScope ls(c, Op::family(), st);
            k_ntt2_first<INV, LOGR, Op><<<sp.nunits * ns * t1, kThr2, smem, st>>>(op, c->tabs(), sp, c->d_ntt2);
        }
        {
            LaunchScope ls(c, Op::family(), st);
            k_ntt2_second<INV, LOGR, Op><<<sp.nunits * t2, kThr2, smem, st>>>(op, c->tabs(), sp, c->d_ntt2);
        }
    }
}

template <bool INV, class Op>
static void launch_ntt(const fhe_ctx* c, const Op& op, cudaStream_t st)
{
    const int count = op.count();
    if (count <= 0) return;
    // the two-pass schedule needs the same number of transforms in every unit
    const bool single = c->force_single_pass || !uniform_subs<Op>::value;
    // (callers refuse single-pass-only work above kMaxSinglePassN)
    const int v = single && (c->ntt_variant == 3 || c->ntt_variant == 4) ? 1 : c->ntt_variant;
    switch (v) {
    case 1: launch_ntt_v<INV, 3, 1024>(c, op, count, st); break;
    case 2: launch_ntt_v<INV, 4, 1024>(c, op, count, st); break;
    case 3: launch_ntt_2pass<INV, 4>(c, op, count, st); break;
    case 4: launch_ntt_2pass<INV, 3>(c, op, count, st); break;
    case 5: launch_ntt_v<INV, 5, 512>(c, op, count, st); break;
    default: launch_ntt_v<INV, 4, 512>(c, op, count, st); break;
    }
}

const char* ntt_variant_name(int v)
{
    switch (v) {
    case 1: return "radix-8 passes, 1024 threads";
    case 2: return "radix-16 passes, 1024 threads";
    case 3: return "two-pass column/row tiles, radix-16";
    case 4: return "two-pass column/row tiles, radix-8";
    case 5: return "radix-32 passes, 512 threads";
    default: return "radix-16 passes, 512 threads";
    }
}

// ---------------------------------------------------------------- ops
// in-place / out-of-place transform of rows of polynomials
struct OpRows {
    static const char* family() { return "ntt"; }
    const u64* src;
    u64* dst;
    int n, rows, N;
    uint8_t pmap[64];
    __host__ __device__ int count() const { return n; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int p, int) const { return pmap[p % rows]; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC&) const { return src[(size_t)p * N + j]; }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC&) const { dst[(size_t)p * N + j] = v; }
};

void k_ntt_rows(const fhe_ctx* c, u64* d, uint32_t n_poly, uint32_t rows, const uint8_t* row_prime, bool forward,
                cudaStream_t st)
{
    OpRows op;
    op.src = d;
    op.dst = d;
    op.n = (int)(n_poly * rows);
    op.rows = (int)rows;
    op.N = (int)c->N;
    for (uint32_t r = 0; r < rows && r < 64; ++r) op.pmap[r] = row_prime[r];
    if (forward) launch_ntt<false>(c, op, st);
    else launch_ntt<true>(c, op, st);
}

void k_ct_to_coeff(const fhe_ctx* c, const u64* in, u64* out, uint32_t n_ct, uint32_t comps, uint32_t L, bool to_coeff,
                   cudaStream_t st)
{
    OpRows op;
    op.src = in;
    op.dst = out;
    op.n = (int)(n_ct * comps * L);
    op.rows = (int)L;
    op.N = (int)c->N;
    for (uint32_t r = 0; r < L; ++r) op.pmap[r] = (uint8_t)r;
    if (to_coeff) launch_ntt<true>(c, op, st);
    else launch_ntt<false>(c, op, st);
}

// ---------------------------------------------------------------- element-wise
// per-prime constants for element-wise kernels come from the resident table
__global__ void k_add_kernel(const u64* __restrict__ a, const u64* __restrict__ b, u64* __restrict__ out,
                             size_t total, int L, int logN, const PrimeC* __restrict__ pc)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)((i >> logN) % L);
        const u64 q = pc[r].q;
        out[i] = add_mod(a[i], b[i], q);
    }
}

static int ew_grid(size_t total)
{
    size_t g = (total + 255) / 256;
    return (int)std::min<size_t>(g, 152 * 32);
}

void k_add(const fhe_ctx* c, const u64* a, const u64* b, u64* out, uint32_t n_ct, uint32_t comps, uint32_t L,
           cudaStream_t st)
{
    size_t total = (size_t)n_ct * comps * L * c->N;
    if (!total) return;
    LaunchScope ls(c, "elementwise", st);
    k_add_kernel<<<ew_grid(total), 256, 0, st>>>(a, b, out, total, (int)L, (int)c->logN, c->d_pc);
}

__global__ void k_tensor_kernel(const u64* __restrict__ a, const u64* __restrict__ b, u64* __restrict__ out,
                                size_t per_comp, int n_ct, int L, int logN, const PrimeC* __restrict__ pc)
{
    // per_comp = L * N; thread covers (ct, r, j)
    const size_t total = (size_t)n_ct * per_comp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t ct = i / per_comp, w = i % per_comp;
        const int r = (int)(w >> logN);
        const PrimeC P = pc[r];
        const u64* A = a + ct * 2 * per_comp;
        const u64* B = b + ct * 2 * per_comp;
        const u64 a0 = A[w], a1 = A[per_comp + w], b0 = B[w], b1 = B[per_comp + w];
        u64* O = out + ct * 3 * per_comp;
        O[w] = mul_mod(a0, b0, P);
        O[per_comp + w] = add_mod(mul_mod(a0, b1, P), mul_mod(a1, b0, P), P.q);
        O[2 * per_comp + w] = mul_mod(a1, b1, P);
    }
}

void k_tensor(const fhe_ctx* c, const u64* a, const u64* b, u64* out3, uint32_t n_ct, uint32_t L, cudaStream_t st)
{
    const size_t per_comp = (size_t)L * c->N;
    const size_t total = (size_t)n_ct * per_comp;
    if (!total) return;
    LaunchScope ls(c, "tensor", st);
    k_tensor_kernel<<<ew_grid(total), 256, 0, st>>>(a, b, out3, per_comp, (int)n_ct, (int)L, (int)c->logN, c->d_pc);
}

// cres[ct * cstride + r]: residues of one integer constant per ciphertext
// (cstride = 0: one constant for all).  Reads residues r < L_out of an input
// stored with L_in residues (L_out < L_in is a mod-drop on the fly).
__global__ void k_mul_const_kernel(const u64* __restrict__ in, u64* __restrict__ out, size_t total, int comps, int L_in,
                                   int L_out, int logN, const u64* __restrict__ cres, int cstride,
                                   const PrimeC* __restrict__ pc)
{
    const size_t Nm = ((size_t)1 << logN) - 1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i >> logN;            // (ct, comp, r) with r < L_out
        const int r = (int)(row % L_out);
        const size_t poly = row / L_out;
        const size_t ct = poly / comps;
        const PrimeC P = pc[r];
        const u64 x = in[((poly * L_in + r) << logN) + (i & Nm)];
        out[i] = mul_mod(x, cres[ct * cstride + r], P);
    }
}

void k_mul_const(const fhe_ctx* c, const u64* in, u64* out, uint32_t n_ct, uint32_t comps, uint32_t L_in, uint32_t L_out,
                 const u64* cres, uint32_t cstride, cudaStream_t st)
{
    size_t total = (size_t)n_ct * comps * L_out * c->N;
    if (!total) return;
    LaunchScope ls(c, "elementwise", st);
    k_mul_const_kernel<<<ew_grid(total), 256, 0, st>>>(in, out, total, (int)comps, (int)L_in, (int)L_out, (int)c->logN,
                                                       cres, (int)cstride, c->d_pc);
}

// constant polynomial (C, 0, ..., 0) is C at every NTT point: add to comp 0
__global__ void k_add_const_kernel(u64* __restrict__ ct, size_t total, int L, int logN, const u64* __restrict__ cres,
                                   int cstride, const PrimeC* __restrict__ pc)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i >> logN;                // (ct, r) over comp 0 only
        const size_t n = row / L;
        const int r = (int)(row % L);
        const size_t idx = (n * 2 * L + r) * ((size_t)1 << logN) + (i & (((size_t)1 << logN) - 1));
        ct[idx] = add_mod(ct[idx], cres[n * cstride + r], pc[r].q);
    }
}

void k_add_const(const fhe_ctx* c, u64* ct, uint32_t n_ct, uint32_t L, const u64* cres, uint32_t cstride, cudaStream_t st)
{
    size_t total = (size_t)n_ct * L * c->N;
    if (!total) return;
    LaunchScope ls(c, "elementwise", st);
    k_add_const_kernel<<<ew_grid(total), 256, 0, st>>>(ct, total, (int)L, (int)c->logN, cres, (int)cstride, c->d_pc);
}

// T = t1 + x2 * c2 + x|_{L1} * c1 over L1 residues (x stored with Lx residues):
// the sum of the three terms of the degree-3 activation in one pass
__global__ void k_poly_combine_kernel(u64* __restrict__ t1, const u64* __restrict__ x2, const u64* __restrict__ x,
                                      size_t total, int L1, int Lx, int logN, const u64* __restrict__ c2,
                                      const u64* __restrict__ c1, const PrimeC* __restrict__ pc)
{
    const size_t Nm = ((size_t)1 << logN) - 1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i >> logN;            // (ct, comp, r), r < L1
        const int r = (int)(row % L1);
        const size_t poly = row / L1;
        const PrimeC P = pc[r];
        const u64 xv = x[((poly * Lx + r) << logN) + (i & Nm)];
        u64 a = add_mod(t1[i], mul_mod(x2[i], c2[r], P), P.q);
        t1[i] = add_mod(a, mul_mod(xv, c1[r], P), P.q);
    }
}

void k_poly_combine(const fhe_ctx* c, u64* t1, const u64* x2, const u64* x, uint32_t n_ct, uint32_t L1, uint32_t Lx,
                    const u64* c2, const u64* c1, cudaStream_t st)
{
    const size_t total = (size_t)n_ct * 2 * L1 * c->N;
    if (!total) return;
    LaunchScope ls(c, "elementwise", st);
    k_poly_combine_kernel<<<ew_grid(total), 256, 0, st>>>(t1, x2, x, total, (int)L1, (int)Lx, (int)c->logN, c2, c1,
                                                          c->d_pc);
}

// ---------------------------------------------------------------- rescale
DivC make_divc(const fhe_ctx* c, uint32_t p_index, uint32_t n_targets)
{
    DivC d;
    const u64 p = c->primes[p_index];
    d.p = p;
    d.p_half = (p - 1) / 2;
    for (uint32_t i = 0; i < n_targets && i < 32; ++i) {
        const u64 q = c->primes[i];
        d.inv[i] = hinv(p % q, q);
        d.invs[i] = shoup(d.inv[i], q);
        d.pmod[i] = p % q;
    }
    return d;
}

// INTT of one residue row per (ct, comp) into scratch V (coefficient form)
struct OpTakeRowInv {
    static const char* family() { return "rescale_intt"; }
    const u64* in;
    u64* V;
    int n, L, row, N, pidx;
    const u64* mulc;    // optional: the input is first multiplied by this per-residue constant
    __host__ __device__ int count() const { return n; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int, int) const { return pidx; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& P) const
    {
        const u64 x = in[((size_t)p * L + row) * N + j];
        return mulc ? mul_mod(x, mulc[row], P) : x;
    }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC&) const { V[(size_t)p * N + j] = v; }
};

// out_i = (in_i - NTT([v]_{q_i})) * p^{-1} (+ addc on comp 0)
struct OpDivFwd {
    static const char* family() { return "rescale_ntt"; }
    const u64* in;      // [n_poly][L_in][N]
    const u64* V;       // [n_poly][N]  coefficient form mod p
    u64* out;           // [n_poly][L_out][N]
    const u64* addc;    // optional: residues of a constant added to comp 0, [n_ct][addc_stride]
    int n_poly, comps, L_in, L_out, N, addc_stride;
    const u64* mulc;    // optional: the input is first multiplied by this per-residue constant
    DivC d;
    __host__ __device__ int count() const { return n_poly * L_out; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int p, int) const { return p % L_out; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& Q) const
    {
        const int poly = p / L_out, i = p % L_out;
        return centred_to(V[(size_t)poly * N + j], d.p, d.p_half, d.pmod[i], Q);
    }
    struct Pre { u64 x, c; };
    __device__ Pre pre(int p, int, int j) const
    {
        const int poly = p / L_out, i = p % L_out;
        Pre r;
        r.x = in[((size_t)poly * L_in + i) * N + j];
        r.c = (addc && (poly % comps) == 0) ? addc[(size_t)(poly / comps) * addc_stride + i] : 0;
        return r;
    }
    __device__ void store(int p, int, int j, u64 v, const Pre& pr, const PrimeC& Q) const
    {
        const int poly = p / L_out, i = p % L_out;
        const u64 x = mulc ? mul_mod(pr.x, mulc[i], Q) : pr.x;
        const u64 r = mul_shoup(sub_mod(x, v, Q.q), d.inv[i], d.invs[i], Q.q);
        out[((size_t)poly * L_out + i) * N + j] = add_mod(r, pr.c, Q.q);
    }
};

size_t rescale_scratch_bytes(const fhe_ctx* c, uint32_t n_ct, uint32_t comps)
{
    return (size_t)n_ct * comps * c->N * sizeof(u64);
}

void k_rescale(const fhe_ctx* c, const u64* in, u64* out, uint32_t n_ct, uint32_t comps, uint32_t L, const u64* addc,
               uint32_t addc_stride, void* scratch, cudaStream_t st, const u64* mulc)
{
    if (n_ct == 0) return;
    u64* V = (u64*)scratch;
    OpTakeRowInv a;
    a.in = in;
    a.V = V;
    a.n = (int)(n_ct * comps);
    a.L = (int)L;
    a.row = (int)L - 1;
    a.N = (int)c->N;
    a.pidx = (int)L - 1;
    a.mulc = mulc;
    launch_ntt<true>(c, a, st);
    OpDivFwd b;
    b.in = in;
    b.V = V;
    b.out = out;
    b.addc = addc;
    b.addc_stride = (int)addc_stride;
    b.n_poly = (int)(n_ct * comps);
    b.comps = (int)comps;
    b.L_in = (int)L;
    b.L_out = (int)L - 1;
    b.N = (int)c->N;
    b.d = make_divc(c, L - 1, L - 1);
    b.mulc = mulc;
    launch_ntt<false>(c, b, st);
}

// ---------------------------------------------------------------- relinearise
// step 1: digits D_j = INTT(d2_j) in [0, q_j)
struct OpDigitsInv {
    static const char* family() { return "keyswitch_intt"; }
    const u64* d3;      // [n][3][L][N]
    u64* D;             // [n][L][N]
    int n, L, N;
    __host__ __device__ int count() const { return n * L; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int p, int) const { return p % L; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC&) const
    {
        const int ct = p / L, r = p % L;
        return d3[(((size_t)ct * 3 + 2) * L + r) * N + j];
    }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC&) const { D[(size_t)p * N + j] = v; }
};

// step 2: per (ct, target t in 0..L, t = L meaning P): for every digit u,
// NTT(D_u mod q_t) * ksk_u[k][t], accumulated over u into acc[ct][k][t].
// Keys carry their Shoup quotients, so each key product is one Shoup product.
struct OpModUpMac {
    static const char* family() { return "keyswitch_modup_mac"; }
    const u64* d3;
    const u64* D;
    const ulonglong2* ksk;  // [L_top][2][L_top+1][N] (k, floor(k 2^64 / q))
    u64* acc;               // [n][2][L+1][N]
    int n, L, N, Ltop;
    __host__ __device__ int count() const { return n * (L + 1); }
    __host__ __device__ int nsub(int) const { return L; }
    __device__ int prime(int p, int) const
    {
        const int t = p % (L + 1);
        return t == L ? Ltop : t;
    }
    __device__ bool direct(int p, int u) const { return (p % (L + 1)) == u; }
    __device__ u64 load(int p, int u, int j, const PrimeC& Q) const
    {
        const int ct = p / (L + 1);
        return reduce64(D[((size_t)ct * L + u) * N + j], Q);
    }
    struct Pre {
        ulonglong2 k0, k1;
        u64 a0, a1, dv;
    };
    __device__ Pre pre(int p, int u, int j) const
    {
        const int ct = p / (L + 1), t = p % (L + 1);
        const int tk = t == L ? Ltop : t;
        Pre r;
        r.k0 = __ldg(&ksk[(((size_t)u * 2 + 0) * (Ltop + 1) + tk) * N + j]);
        r.k1 = __ldg(&ksk[(((size_t)u * 2 + 1) * (Ltop + 1) + tk) * N + j]);
        if (u > 0) {
            r.a0 = acc[(((size_t)ct * 2 + 0) * (L + 1) + t) * N + j];
            r.a1 = acc[(((size_t)ct * 2 + 1) * (L + 1) + t) * N + j];
        } else {
            r.a0 = r.a1 = 0;
        }
        r.dv = (t == u) ? d3[(((size_t)ct * 3 + 2) * L + t) * N + j] : 0;   // NTT(d2_t) is d2_t
        return r;
    }
    __device__ void store(int p, int u, int j, u64 v, const Pre& pr, const PrimeC& Q) const
    {
        const int ct = p / (L + 1), t = p % (L + 1);
        if (t == u) v = pr.dv;
        const u64 p0 = mul_shoup(v, pr.k0.x, pr.k0.y, Q.q);
        const u64 p1 = mul_shoup(v, pr.k1.x, pr.k1.y, Q.q);
        acc[(((size_t)ct * 2 + 0) * (L + 1) + t) * N + j] = u == 0 ? p0 : add_mod(pr.a0, p0, Q.q);
        acc[(((size_t)ct * 2 + 1) * (L + 1) + t) * N + j] = u == 0 ? p1 : add_mod(pr.a1, p1, Q.q);
    }
};

// step 3: INTT of the P residue of both accumulators
struct OpAccPInv {
    static const char* family() { return "keyswitch_acc_intt"; }
    const u64* acc;
    u64* Vp;            // [n][2][N]
    int n, L, N, Ltop;
    __host__ __device__ int count() const { return n * 2; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int, int) const { return Ltop; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC&) const { return acc[((size_t)p * (L + 1) + L) * N + j]; }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC&) const { Vp[(size_t)p * N + j] = v; }
};

// step 4: ModDown + add: out_k,t = d_k,t + (acc_k,t - NTT([v]_{q_t})) * P^{-1}
struct OpModDown {
    static const char* family() { return "keyswitch_moddown"; }
    const u64* d3;
    const u64* acc;
    const u64* Vp;
    u64* out;           // [n][2][L][N]
    int n, L, N;
    DivC d;
    __host__ __device__ int count() const { return n * 2 * L; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int p, int) const { return p % L; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& Q) const
    {
        const int poly = p / L, t = p % L;             // poly = ct*2 + k
        return centred_to(Vp[(size_t)poly * N + j], d.p, d.p_half, d.pmod[t], Q);
    }
    struct Pre { u64 a, dk; };
    __device__ Pre pre(int p, int, int j) const
    {
        const int poly = p / L, t = p % L;
        const int ct = poly >> 1, k = poly & 1;
        Pre r;
        r.a = acc[((size_t)poly * (L + 1) + t) * N + j];
        r.dk = d3[(((size_t)ct * 3 + k) * L + t) * N + j];
        return r;
    }
    __device__ void store(int p, int, int j, u64 v, const Pre& pr, const PrimeC& Q) const
    {
        const int poly = p / L, t = p % L;
        const int ct = poly >> 1, k = poly & 1;
        const u64 ks = mul_shoup(sub_mod(pr.a, v, Q.q), d.inv[t], d.invs[t], Q.q);
        out[(((size_t)ct * 2 + k) * L + t) * N + j] = add_mod(pr.dk, ks, Q.q);
    }
};

size_t relin_scratch_bytes(const fhe_ctx* c, uint32_t n_ct, uint32_t L)
{
    const size_t N = c->N;
    return arena_need({(size_t)n_ct * L * N * 8, (size_t)n_ct * 2 * (L + 1) * N * 8, (size_t)n_ct * 2 * N * 8});
}

void k_relin(const fhe_ctx* c, const u64* d3, u64* out2, uint32_t n_ct, uint32_t L, void* scratch, cudaStream_t st)
{
    if (n_ct == 0) return;
    const size_t N = c->N;
    Arena ar;
    ar.base = (char*)scratch;
    ar.cap = relin_scratch_bytes(c, n_ct, L);
    u64* D = (u64*)ar.take((size_t)n_ct * L * N * 8);
    u64* acc = (u64*)ar.take((size_t)n_ct * 2 * (L + 1) * N * 8);
    u64* Vp = (u64*)ar.take((size_t)n_ct * 2 * N * 8);

    OpDigitsInv s1{d3, D, (int)n_ct, (int)L, (int)N};
    launch_ntt<true>(c, s1, st);
    OpModUpMac s2{d3, D, c->d_ksk, acc, (int)n_ct, (int)L, (int)N, (int)c->L_top};
    launch_ntt<false>(c, s2, st);
    OpAccPInv s3{acc, Vp, (int)n_ct, (int)L, (int)N, (int)c->L_top};
    launch_ntt<true>(c, s3, st);
    OpModDown s4;
    s4.d3 = d3;
    s4.acc = acc;
    s4.Vp = Vp;
    s4.out = out2;
    s4.n = (int)n_ct;
    s4.L = (int)L;
    s4.N = (int)N;
    s4.d = make_divc(c, c->L_top, L);
    launch_ntt<false>(c, s4, st);
}

// ---------------------------------------------------------------- level groups
// ct-mult + relinearise + rescale for batches at different levels: every step
// is one launch over all batches (MultiOp), so a set of uneven-level
// ciphertexts costs seven launches whatever its level mix.
struct TensorGroups {
    const u64* a[kMaxGroups];
    const u64* b[kMaxGroups];
    u64* out[kMaxGroups];
    unsigned long long start[kMaxGroups + 1];
    int L[kMaxGroups];
    int ng;
};

__global__ void k_tensor_groups_kernel(TensorGroups G, int logN, const PrimeC* __restrict__ pc)
{
    const size_t total = G.start[G.ng];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        int g = 0;
        while (g + 1 < G.ng && i >= G.start[g + 1]) ++g;
        const size_t w0 = i - G.start[g];
        const size_t per_comp = (size_t)G.L[g] << logN;
        const size_t ct = w0 / per_comp, w = w0 % per_comp;
        const int r = (int)(w >> logN);
        const PrimeC P = pc[r];
        const u64* A = G.a[g] + ct * 2 * per_comp;
        const u64* B = G.b[g] + ct * 2 * per_comp;
        const u64 a0 = A[w], a1 = A[per_comp + w], b0 = B[w], b1 = B[per_comp + w];
        u64* O = G.out[g] + ct * 3 * per_comp;
        O[w] = mul_mod(a0, b0, P);
        O[per_comp + w] = add_mod(mul_mod(a0, b1, P), mul_mod(a1, b0, P), P.q);
        O[2 * per_comp + w] = mul_mod(a1, b1, P);
    }
}

size_t level_groups_scratch_bytes(const fhe_ctx* c, const LevelBatch* g, int ng)
{
    const size_t N = c->N;
    size_t s = 0;
    for (int k = 0; k < ng; ++k) {
        const size_t n = g[k].n, L = g[k].L;
        s += arena_need({n * 3 * L * N * 8, n * 2 * L * N * 8, n * L * N * 8, n * 2 * (L + 1) * N * 8,
                         n * 2 * N * 8, n * 2 * N * 8});
    }
    return s;
}

void k_mul_relin_rescale_groups(const fhe_ctx* c, const LevelBatch* g, int ng, void* scratch, cudaStream_t st)
{
    const size_t N = c->N;
    Arena ar;
    ar.base = (char*)scratch;
    ar.cap = level_groups_scratch_bytes(c, g, ng);
    TensorGroups tg;
    MultiOp<OpDigitsInv> m1;
    MultiOp<OpModUpMac> m2;
    MultiOp<OpAccPInv> m3;
    MultiOp<OpModDown> m4;
    MultiOp<OpTakeRowInv> m5;
    MultiOp<OpDivFwd> m6;
    m1.ng = m2.ng = m3.ng = m4.ng = m5.ng = m6.ng = tg.ng = ng;
    m1.pre_[0] = m2.pre_[0] = m3.pre_[0] = m4.pre_[0] = m5.pre_[0] = m6.pre_[0] = 0;
    tg.start[0] = 0;
    for (int k = 0; k < ng; ++k) {
        const int n = (int)g[k].n, L = (int)g[k].L;
        u64* t3 = (u64*)ar.take((size_t)n * 3 * L * N * 8);
        u64* t2 = (u64*)ar.take((size_t)n * 2 * L * N * 8);
        u64* D = (u64*)ar.take((size_t)n * L * N * 8);
        u64* acc = (u64*)ar.take((size_t)n * 2 * (L + 1) * N * 8);
        u64* Vp = (u64*)ar.take((size_t)n * 2 * N * 8);
        u64* V = (u64*)ar.take((size_t)n * 2 * N * 8);
        tg.a[k] = g[k].a;
        tg.b[k] = g[k].b;
        tg.out[k] = t3;
        tg.L[k] = L;
        tg.start[k + 1] = tg.start[k] + (unsigned long long)n * L * N;
        m1.ops[k] = OpDigitsInv{t3, D, n, L, (int)N};
        m2.ops[k] = OpModUpMac{t3, D, c->d_ksk, acc, n, L, (int)N, (int)c->L_top};
        m3.ops[k] = OpAccPInv{acc, Vp, n, L, (int)N, (int)c->L_top};
        OpModDown md;
        md.d3 = t3;
        md.acc = acc;
        md.Vp = Vp;
        md.out = t2;
        md.n = n;
        md.L = L;
        md.N = (int)N;
        md.d = make_divc(c, c->L_top, L);
        m4.ops[k] = md;
        OpTakeRowInv tr;
        tr.in = t2;
        tr.V = V;
        tr.n = n * 2;
        tr.L = L;
        tr.row = L - 1;
        tr.N = (int)N;
        tr.pidx = L - 1;
        tr.mulc = nullptr;
        m5.ops[k] = tr;
        OpDivFwd dv;
        dv.in = t2;
        dv.V = V;
        dv.out = g[k].out;
        dv.addc = nullptr;
        dv.addc_stride = 0;
        dv.n_poly = n * 2;
        dv.comps = 2;
        dv.L_in = L;
        dv.L_out = L - 1;
        dv.N = (int)N;
        dv.d = make_divc(c, L - 1, L - 1);
        dv.mulc = nullptr;
        m6.ops[k] = dv;
        m1.pre_[k + 1] = m1.pre_[k] + m1.ops[k].count();
        m2.pre_[k + 1] = m2.pre_[k] + m2.ops[k].count();
        m3.pre_[k + 1] = m3.pre_[k] + m3.ops[k].count();
        m4.pre_[k + 1] = m4.pre_[k] + m4.ops[k].count();
        m5.pre_[k + 1] = m5.pre_[k] + m5.ops[k].count();
        m6.pre_[k + 1] = m6.pre_[k] + m6.ops[k].count();
    }
    {
        LaunchScope ls(c, "tensor", st);
        k_tensor_groups_kernel<<<ew_grid(tg.start[ng]), 256, 0, st>>>(tg, (int)c->logN, c->d_pc);
    }
    launch_ntt<true>(c, m1, st);
    launch_ntt<false>(c, m2, st);
    launch_ntt<true>(c, m3, st);
    launch_ntt<false>(c, m4, st);
    launch_ntt<true>(c, m5, st);
    launch_ntt<false>(c, m6, st);
}

// ---------------------------------------------------------------- linear layers
// Y[o][k][r][j] = sum_{e in row o} W[e][r] * X[col[e]][k][r][j]  (mod q_r)
// grid: x = output o (fastest, so outputs sharing inputs run together and
// reuse the input slice from L2), y = coefficient block, z = k * L + r.
__global__ void __launch_bounds__(256) k_mac_kernel(const u64* __restrict__ X, const uint32_t* __restrict__ row_ptr,
                                                     const uint32_t* __restrict__ col, const u64* __restrict__ W,
                                                     u64* __restrict__ Y, int L, int N, const PrimeC* __restrict__ pc)
{
    const int o = blockIdx.x;
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    const int kr = blockIdx.z;
    const int r = kr % L;
    if (j >= N) return;
    const PrimeC P = pc[r];
    const size_t ct_stride = (size_t)2 * L * N;
    const size_t off = (size_t)kr * N + j;
    const uint32_t e0 = row_ptr[o], e1 = row_ptr[o + 1];
    u64 lo = 0, hi = 0;
    int cnt = 0;
    for (uint32_t e = e0; e < e1; ++e) {
        const u64 x = X[(size_t)col[e] * ct_stride + off];
        const u64 w = W[(size_t)e * L + r];
        const u64 pl = x * w, ph = __umul64hi(x, w);
        lo += pl;
        hi += ph + (lo < pl ? 1 : 0);
        if (++cnt == 32) {              // hi < 32 * 2^58: fold before it can overflow
            lo = reduce128(hi, lo, P);
            hi = 0;
            cnt = 0;
        }
    }
    Y[(size_t)o * ct_stride + off] = reduce128(hi, lo, P);
}

void k_linear_mac(const fhe_ctx* c, const u64* X, uint32_t n_in, const uint32_t* row_ptr, const uint32_t* col,
                  const u64* Wres, uint32_t n_out, uint32_t L, u64* Y, cudaStream_t st)
{
    (void)n_in;
    if (n_out == 0) return;
    const int N = (int)c->N;
    const int tpb = N < 256 ? N : 256;
    dim3 grid(n_out, (N + tpb - 1) / tpb, 2 * L);
    LaunchScope ls(c, "mac", st);
    k_mac_kernel<<<grid, tpb, 0, st>>>(X, row_ptr, col, Wres, Y, (int)L, N, c->d_pc);
}

// Tiled form: rows sharing one column list are computed together, up to
// kMacTile per thread, so each input word is loaded once per tile.
//   tiles[t] = {col_off, K, n_rows, w_off}; rows[t * kMacTile + o] = output row;
//   W[((w_off + e) * L + r) * kMacTile + o] = weight residue of (row o, term e)
// (the tile's weights of one term and residue are contiguous: 4 vector loads).
// Terms are processed four at a time with their input loads issued together.
__device__ __forceinline__ void mac128(u64& lo, u64& hi, u64 x, u64 w)
{
    const u64 pl = x * w, ph = __umul64hi(x, w);
    lo += pl;
    hi += ph + (lo < pl ? 1 : 0);
}

// Limb form for primes below 2^42: x = xH 2^21 + xL and the stored weight
// word holds wL | wH << 32 with w = wH 2^21 + wL (all limbs < 2^21), so every
// limb product is < 2^42 and accumulates exactly in a 64-bit register with one
// 32 x 32 + 64 multiply-add: sum x w = S0 + S1 2^21 + S2 2^42 with
// S0 = sum xL wL, S1 = sum (xL wH + xH wL), S2 = sum xH wH (no carries for
// fewer than 2^20 terms).
constexpr u64 kLimbMask = (1ull << 21) - 1;

__device__ __forceinline__ u64 limb_combine(u64 s0, u64 s1, u64 s2, const PrimeC& P)
{
    u64 lo = s0 + (s1 << 21);
    u64 hi = (s1 >> 43) + (lo < s0 ? 1 : 0);
    const u64 t = s2 << 42;
    lo += t;
    hi += (s2 >> 22) + (lo < t ? 1 : 0);
    return reduce128(hi, lo, P);
}

__global__ void __launch_bounds__(256) k_mac_tiled_kernel(const u64* __restrict__ X, const uint4* __restrict__ tiles,
                                                           const uint32_t* __restrict__ rows,
                                                           const uint32_t* __restrict__ col,
                                                           const u64* __restrict__ W, u64* __restrict__ Y, int L, int N,
                                                           const PrimeC* __restrict__ pc)
{
    const uint4 tl = tiles[blockIdx.x];
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    const int kr = blockIdx.z;
    const int r = kr % L;
    if (j >= N) return;
    const PrimeC P = pc[r];
    const size_t ct_stride = (size_t)2 * L * N;
    const u64* Xj = X + (size_t)kr * N + j;
    const uint32_t* cl = col + tl.x;
    const ulonglong2* w2 = reinterpret_cast<const ulonglong2*>(W + ((size_t)tl.w * L + r) * kMacTile);
    const size_t wstep = (size_t)L * kMacTile / 2;        // ulonglong2 per term
    const size_t off = (size_t)kr * N + j;
    const uint32_t K = tl.y;
    if (P.q < kLimbPrimeBound) {                            // block-uniform branch
        u64 s0[kMacTile], s1[kMacTile], s2[kMacTile];
#pragma unroll
        for (int o = 0; o < kMacTile; ++o) s0[o] = s1[o] = s2[o] = 0;
        uint32_t e = 0;
        for (; e + 4 <= K; e += 4) {
            u64 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = Xj[(size_t)__ldg(&cl[e + u]) * ct_stride];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t xl = (uint32_t)(x[u] & kLimbMask), xh = (uint32_t)(x[u] >> 21);
                const ulonglong2* we = w2 + (size_t)(e + u) * wstep;
#pragma unroll
                for (int o2 = 0; o2 < kMacTile / 2; ++o2) {
                    const ulonglong2 wv = __ldg(&we[o2]);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const u64 wd = h ? wv.y : wv.x;
                        const uint32_t wl = (uint32_t)wd, wh = (uint32_t)(wd >> 32);
                        const int o = 2 * o2 + h;
                        s0[o] += (u64)xl * wl;
                        s1[o] += (u64)xl * wh;
                        s1[o] += (u64)xh * wl;
                        s2[o] += (u64)xh * wh;
                    }
                }
            }
        }
        for (; e < K; ++e) {
            const u64 xv = Xj[(size_t)__ldg(&cl[e]) * ct_stride];
            const uint32_t xl = (uint32_t)(xv & kLimbMask), xh = (uint32_t)(xv >> 21);
            const ulonglong2* we = w2 + (size_t)e * wstep;
#pragma unroll
            for (int o2 = 0; o2 < kMacTile / 2; ++o2) {
                const ulonglong2 wv = __ldg(&we[o2]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const u64 wd = h ? wv.y : wv.x;
                    const uint32_t wl = (uint32_t)wd, wh = (uint32_t)(wd >> 32);
                    const int o = 2 * o2 + h;
                    s0[o] += (u64)xl * wl;
                    s1[o] += (u64)xl * wh;
                    s1[o] += (u64)xh * wl;
                    s2[o] += (u64)xh * wh;
                }
            }
        }
#pragma unroll
        for (int o = 0; o < kMacTile; ++o)
            if (o < (int)tl.z)
                Y[(size_t)rows[blockIdx.x * kMacTile + o] * ct_stride + off] = limb_combine(s0[o], s1[o], s2[o], P);
        return;
    }
    u64 lo[kMacTile], hi[kMacTile];
#pragma unroll
    for (int o = 0; o < kMacTile; ++o) lo[o] = hi[o] = 0;
    uint32_t e = 0;
    int cnt = 0;
    for (; e + 4 <= K; e += 4) {
        u64 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = Xj[(size_t)__ldg(&cl[e + u]) * ct_stride];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const ulonglong2* we = w2 + (size_t)(e + u) * wstep;
#pragma unroll
            for (int o2 = 0; o2 < kMacTile / 2; ++o2) {
                const ulonglong2 wv = __ldg(&we[o2]);
                mac128(lo[2 * o2], hi[2 * o2], x[u], wv.x);
                mac128(lo[2 * o2 + 1], hi[2 * o2 + 1], x[u], wv.y);
            }
        }
        cnt += 4;
        if (cnt == 32) {                // hi < 32 * 2^58: fold before it can overflow
#pragma unroll
            for (int o = 0; o < kMacTile; ++o) {
                lo[o] = reduce128(hi[o], lo[o], P);
                hi[o] = 0;
            }
            cnt = 0;
        }
    }
    for (; e < K; ++e) {
        const u64 x = Xj[(size_t)__ldg(&cl[e]) * ct_stride];
        const ulonglong2* we = w2 + (size_t)e * wstep;
#pragma unroll
        for (int o2 = 0; o2 < kMacTile / 2; ++o2) {
            const ulonglong2 wv = __ldg(&we[o2]);
            mac128(lo[2 * o2], hi[2 * o2], x, wv.x);
            mac128(lo[2 * o2 + 1], hi[2 * o2 + 1], x, wv.y);
        }
    }
#pragma unroll
    for (int o = 0; o < kMacTile; ++o)
        if (o < (int)tl.z) Y[(size_t)rows[blockIdx.x * kMacTile + o] * ct_stride + off] = reduce128(hi[o], lo[o], P);
}

void k_linear_mac_tiled(const fhe_ctx* c, const u64* X, const uint4* tiles, uint32_t n_tiles, const uint32_t* rows,
                        const uint32_t* col, const u64* W, uint32_t L, u64* Y, cudaStream_t st)
{
    if (n_tiles == 0) return;
    const int N = (int)c->N;
    const int tpb = N < 256 ? N : 256;
    dim3 grid(n_tiles, (N + tpb - 1) / tpb, 2 * L);
    LaunchScope ls(c, "mac", st);
    k_mac_tiled_kernel<<<grid, tpb, 0, st>>>(X, tiles, rows, col, W, Y, (int)L, N, c->d_pc);
}

// ---------------------------------------------------------------- keys
enum { DOM_SECRET = 1, DOM_PK_A = 2, DOM_PK_E = 3, DOM_KSK_A = 4, DOM_KSK_E = 5,
       DOM_ENC_U = 6, DOM_ENC_E0 = 7, DOM_ENC_E1 = 8 };

// s (ternary) in every key prime
struct OpSecret {
    static const char* family() { return "keygen"; }
    u64* s;
    u64 s0;
    int nprimes, N;
    __host__ __device__ int count() const { return nprimes; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int p, int) const { return p; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int, int, int j, const PrimeC& P) const { return from_signed(draw_ternary(s0, j), P); }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC&) const { s[(size_t)p * N + j] = v; }
};

// pk = (-a s + e, a) over the data primes: sub 0 = a (uniform), sub 1 = e
struct OpPublicKey {
    static const char* family() { return "keygen"; }
    const u64* s;
    u64* pk;            // [2][Ltop][N]
    const u64* cdt;
    u64 sa, se;
    int Ltop, N;
    __host__ __device__ int count() const { return Ltop; }
    __host__ __device__ int nsub(int) const { return 2; }
    __device__ int prime(int p, int) const { return p; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int u, int j, const PrimeC& P) const
    {
        return u == 0 ? draw_uniform(sa, j, p, P) : from_signed(draw_gauss(se, j, cdt), P);
    }
    struct Pre { u64 x; };
    __device__ Pre pre(int p, int u, int j) const
    {
        return {u == 0 ? s[(size_t)p * N + j] : pk[(size_t)p * N + j]};
    }
    __device__ void store(int p, int u, int j, u64 v, const Pre& pr, const PrimeC& P) const
    {
        u64* b = pk + (size_t)p * N;
        u64* a = pk + ((size_t)Ltop + p) * N;
        if (u == 0) {
            a[j] = v;
            b[j] = sub_mod(0, mul_mod(v, pr.x, P), P.q);
        } else {
            b[j] = add_mod(pr.x, v, P.q);
        }
    }
};

// ksk_j = (-a_j s + e_j + [r == j] P s^2, a_j) over every key prime r; each
// key word is stored with its Shoup quotient floor(k 2^64 / q)
__device__ __forceinline__ ulonglong2 with_shoup(u64 k, u64 q)
{
    return make_ulonglong2(k, (u64)(((unsigned __int128)k << 64) / q));
}

struct OpRelinKey {
    static const char* family() { return "keygen"; }
    const u64* s;
    ulonglong2* ksk;    // [Ltop][2][Ltop+1][N]
    const u64* cdt;
    const u64* sa;      // per digit stream keys (device array [Ltop])
    const u64* se;
    u64 Pmod[33];       // P mod q_r
    int Ltop, N;
    __host__ __device__ int count() const { return Ltop * (Ltop + 1); }
    __host__ __device__ int nsub(int) const { return 2; }
    __device__ int prime(int p, int) const { return p % (Ltop + 1); }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int u, int j, const PrimeC& P) const
    {
        const int dj = p / (Ltop + 1), r = p % (Ltop + 1);
        return u == 0 ? draw_uniform(sa[dj], j, r, P) : from_signed(draw_gauss(se[dj], j, cdt), P);
    }
    struct Pre { u64 sr, b; };
    __device__ Pre pre(int p, int u, int j) const
    {
        const int dj = p / (Ltop + 1), r = p % (Ltop + 1);
        Pre x;
        x.sr = s[(size_t)r * N + j];
        x.b = u == 1 ? ksk[(((size_t)dj * 2 + 0) * (Ltop + 1) + r) * N + j].x : 0;
        return x;
    }
    __device__ void store(int p, int u, int j, u64 v, const Pre& pr, const PrimeC& P) const
    {
        const int dj = p / (Ltop + 1), r = p % (Ltop + 1);
        ulonglong2* b = ksk + (((size_t)dj * 2 + 0) * (Ltop + 1) + r) * N;
        ulonglong2* a = ksk + (((size_t)dj * 2 + 1) * (Ltop + 1) + r) * N;
        if (u == 0) {
            a[j] = with_shoup(v, P.q);
            b[j] = make_ulonglong2(sub_mod(0, mul_mod(v, pr.sr, P), P.q), 0);
        } else {
            u64 x = add_mod(pr.b, v, P.q);
            if (r == dj) x = add_mod(x, mul_mod(Pmod[r], mul_mod(pr.sr, pr.sr, P), P), P.q);
            b[j] = with_shoup(x, P.q);
        }
    }
};

void k_keygen(fhe_ctx* c, cudaStream_t st)
{
    const int N = (int)c->N, Lt = (int)c->L_top;
    OpSecret os{c->d_s, stream_key(c->seed, DOM_SECRET, 0), Lt + 1, N};
    launch_ntt<false>(c, os, st);
    OpPublicKey op{c->d_s, c->d_pk, c->d_cdt, stream_key(c->seed, DOM_PK_A, 0), stream_key(c->seed, DOM_PK_E, 0), Lt, N};
    launch_ntt<false>(c, op, st);
    std::vector<u64> h(2 * Lt);
    for (int j = 0; j < Lt; ++j) {
        h[j] = stream_key(c->seed, DOM_KSK_A, (u64)j);
        h[Lt + j] = stream_key(c->seed, DOM_KSK_E, (u64)j);
    }
    u64* dkeys = nullptr;
    cudaMallocAsync((void**)&dkeys, h.size() * 8, st);
    cudaMemcpyAsync(dkeys, h.data(), h.size() * 8, cudaMemcpyHostToDevice, st);
    OpRelinKey ok;
    ok.s = c->d_s;
    ok.ksk = c->d_ksk;
    ok.cdt = c->d_cdt;
    ok.sa = dkeys;
    ok.se = dkeys + Lt;
    for (int r = 0; r <= Lt && r < 33; ++r) ok.Pmod[r] = c->primes[Lt] % c->primes[r];
    ok.Ltop = Lt;
    ok.N = N;
    launch_ntt<false>(c, ok, st);
    cudaFreeAsync(dkeys, st);
}

// ---------------------------------------------------------------- encrypt
// The integer samples of a ciphertext (u, e0, e1) are drawn once per
// coefficient by k_sample_enc (int8, [n][3][N]) and then reduced into every
// residue by the transform prologue.
__device__ __forceinline__ i64 draw_gauss_bs(u64 s0, int j, const u64* __restrict__ cdt)
{
    const u64 u = sm_out(s0, (u64)j);
    int lo = 0, hi = 38;                 // number of thresholds <= u (table increasing)
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&cdt[mid]) <= u) lo = mid + 1;
        else hi = mid;
    }
    return (i64)lo - 19;
}

__global__ void k_sample_enc_kernel(int8_t* __restrict__ S, int n, int N, u64 seed, u64 first,
                                    const u64* __restrict__ cdt)
{
    const size_t total = (size_t)n * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ci = (int)(i / N), j = (int)(i % N);
        const u64 id = first + (u64)ci;
        int8_t* o = S + (size_t)ci * 3 * N + j;
        o[0] = (int8_t)draw_ternary(sm_out(sm_out(seed, (u64)DOM_ENC_U), id), j);
        o[N] = (int8_t)draw_gauss_bs(sm_out(sm_out(seed, (u64)DOM_ENC_E0), id), j, cdt);
        o[2 * (size_t)N] = (int8_t)draw_gauss_bs(sm_out(sm_out(seed, (u64)DOM_ENC_E1), id), j, cdt);
    }
}

// per (ct, r): sub 0 = u, sub 1 = e0, sub 2 = e1
struct OpEncrypt {
    static const char* family() { return "encrypt"; }
    const u64* pt;      // [n][Ltop][N]
    const u64* pk;      // [2][Ltop][N]
    u64* ct;            // [n][2][Ltop][N]
    const int8_t* S;    // [n][3][N] samples
    const i64* M;       // optional [n][N] encoded coefficients (then pt is unused):
                        // NTT(e0) + NTT(m) = NTT(e0 + m), so the plaintext needs no transform of its own
    int n, Ltop, N;
    __host__ __device__ int count() const { return n * Ltop; }
    __host__ __device__ int nsub(int) const { return 3; }
    __device__ int prime(int p, int) const { return p % Ltop; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int u, int j, const PrimeC& P) const
    {
        const int ci = p / Ltop;
        i64 v = (i64)S[((size_t)ci * 3 + u) * N + j];
        if (u == 1 && M) v += M[(size_t)ci * N + j];
        return from_signed(v, P);
    }
    struct Pre { u64 a, b, c; };
    __device__ Pre pre(int p, int u, int j) const
    {
        const int ci = p / Ltop, r = p % Ltop;
        Pre x;
        if (u == 0) {
            x.a = M ? 0 : pt[((size_t)ci * Ltop + r) * N + j];
            x.b = pk[(size_t)r * N + j];
            x.c = pk[((size_t)Ltop + r) * N + j];
        } else {
            x.a = ct[(((size_t)ci * 2 + (u == 1 ? 0 : 1)) * Ltop + r) * N + j];
            x.b = x.c = 0;
        }
        return x;
    }
    __device__ void store(int p, int u, int j, u64 v, const Pre& pr, const PrimeC& P) const
    {
        const int ci = p / Ltop, r = p % Ltop;
        u64* c0 = ct + (((size_t)ci * 2 + 0) * Ltop + r) * N;
        u64* c1 = ct + (((size_t)ci * 2 + 1) * Ltop + r) * N;
        if (u == 0) {
            c0[j] = add_mod(mul_mod(v, pr.b, P), pr.a, P.q);
            c1[j] = mul_mod(v, pr.c, P);
        } else if (u == 1) {
            c0[j] = add_mod(pr.a, v, P.q);
        } else {
            c1[j] = add_mod(pr.a, v, P.q);
        }
    }
};

size_t encrypt_scratch_bytes(const fhe_ctx* c, uint32_t n_ct) { return (size_t)n_ct * 3 * c->N; }

void k_encrypt(const fhe_ctx* c, const u64* pt, uint32_t n_ct, uint64_t first_id, u64* ct, void* scratch,
               cudaStream_t st)
{
    if (n_ct == 0) return;
    int8_t* S = (int8_t*)scratch;
    {
        const size_t total = (size_t)n_ct * c->N;
        LaunchScope ls(c, "encrypt", st);
        k_sample_enc_kernel<<<ew_grid(total), 256, 0, st>>>(S, (int)n_ct, (int)c->N, c->seed, first_id, c->d_cdt);
    }
    OpEncrypt op{pt, c->d_pk, ct, S, nullptr, (int)n_ct, (int)c->L_top, (int)c->N};
    launch_ntt<false>(c, op, st);
}

size_t encode_encrypt_scratch_bytes(const fhe_ctx* c, uint32_t n_ct)
{
    return arena_need({encode_scratch_bytes(c, n_ct), encrypt_scratch_bytes(c, n_ct)});
}

void k_encode_encrypt(const fhe_ctx* c, const double* slots, uint32_t n_ct, double scale, uint64_t first_id, u64* ct,
                      void* scratch, cudaStream_t st)
{
    if (n_ct == 0) return;
    Arena ar;
    ar.base = (char*)scratch;
    ar.cap = encode_encrypt_scratch_bytes(c, n_ct);
    i64* m = (i64*)ar.take(encode_scratch_bytes(c, n_ct));
    int8_t* S = (int8_t*)ar.take(encrypt_scratch_bytes(c, n_ct));
    encode_coefficients(c, slots, n_ct, scale, m, st);
    {
        const size_t total = (size_t)n_ct * c->N;
        LaunchScope ls(c, "encrypt", st);
        k_sample_enc_kernel<<<ew_grid(total), 256, 0, st>>>(S, (int)n_ct, (int)c->N, c->seed, first_id, c->d_cdt);
    }
    OpEncrypt op{nullptr, c->d_pk, ct, S, m, (int)n_ct, (int)c->L_top, (int)c->N};
    launch_ntt<false>(c, op, st);
}

// ---------------------------------------------------------------- decrypt
// prologue: c0 + c1 s at residue 0 (NTT form); INTT; centred lift
struct OpDecrypt {
    static const char* family() { return "decrypt"; }
    const u64* ct;
    const u64* s;
    i64* m;
    int n, L, N;
    __host__ __device__ int count() const { return n; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int, int) const { return 0; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& P) const
    {
        const u64 c0 = ct[(((size_t)p * 2 + 0) * L) * N + j];
        const u64 c1 = ct[(((size_t)p * 2 + 1) * L) * N + j];
        return add_mod(c0, mul_mod(c1, s[j], P), P.q);
    }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC& P) const
    {
        m[(size_t)p * N + j] = v > P.half ? (i64)v - (i64)P.q : (i64)v;
    }
};

void k_decrypt(const fhe_ctx* c, const u64* ct, uint32_t n_ct, uint32_t L, i64* m, cudaStream_t st)
{
    OpDecrypt op{ct, c->d_s, m, (int)n_ct, (int)L, (int)c->N};
    launch_ntt<true>(c, op, st);
}

// ---------------------------------------------------------------- encode
// double-double helpers (explicit _rn intrinsics: never contracted)
struct ddv { double hi, lo; };
__device__ __forceinline__ ddv two_sum(double a, double b)
{
    double s = __dadd_rn(a, b);
    double bb = __dsub_rn(s, a);
    double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ddv fast_two_sum(double a, double b)
{
    double s = __dadd_rn(a, b);
    return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
// double-double sum with one error-free transformation on the high parts
// (relative error ~2^-100 of the operands: the encoder needs ~2^-70)
__device__ __forceinline__ ddv dadd(ddv a, ddv b)
{
    ddv s = two_sum(a.hi, b.hi);
    s.lo = __dadd_rn(s.lo, __dadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ddv dneg(ddv a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ddv dmul(ddv a, ddv b)
{
    double p = __dmul_rn(a.hi, b.hi);
    double e = __fma_rn(a.hi, b.hi, -p);
    e = __dadd_rn(e, __dadd_rn(__dmul_rn(a.hi, b.lo), __dmul_rn(a.lo, b.hi)));
    return fast_two_sum(p, e);
}
struct cddv { ddv re, im; };
__device__ __forceinline__ cddv cadd(cddv a, cddv b) { return {dadd(a.re, b.re), dadd(a.im, b.im)}; }
__device__ __forceinline__ cddv csub(cddv a, cddv b) { return {dadd(a.re, dneg(b.re)), dadd(a.im, dneg(b.im))}; }
__device__ __forceinline__ cddv cmul(cddv a, cddv b)
{
    return {dadd(dmul(a.re, b.re), dneg(dmul(a.im, b.im))), dadd(dmul(a.re, b.im), dmul(a.im, b.re))};
}
__device__ __forceinline__ cddv ld4(const double4& v) { return {{v.x, v.y}, {v.z, v.w}}; }

// round half away from zero of a double-double to int64
__device__ __forceinline__ i64 dd_round(ddv v)
{
    bool neg = v.hi < 0.0 || (v.hi == 0.0 && v.lo < 0.0);
    if (neg) v = dneg(v);
    double f = floor(v.hi);
    double frac = __dadd_rn(__dsub_rn(v.hi, f), v.lo);
    double add = floor(__dadd_rn(frac, 0.5));
    i64 r = (i64)f + (i64)add;
    return neg ? -r : r;
}

// One block per (ct, half h): the N/2-point inverse DFT of the slots (placed
// at l(j) = (5^j mod 2N - 1)/4) is split by its first decimation-in-frequency
// stage; half h runs the N/4-point DFT of its half in shared memory.
// Output: m_k = round(scale * Re c_k), m_{k+N/2} = round(scale * Im c_k),
// c_k = (2/N) zeta^{-k} X_k.
__global__ void __launch_bounds__(512) k_encode_kernel(const double* __restrict__ slots, const uint32_t* __restrict__ slot_of,
                                                        const double4* __restrict__ tw, const double4* __restrict__ twist,
                                                        double scale_over_M, int N, i64* __restrict__ m)
{
    extern __shared__ double4 A[];       // N/4 complex dd values
    const int M = N / 2, H = M / 2;
    const int ct = blockIdx.x >> 1, h = blockIdx.x & 1;
    const double* z = slots + (size_t)ct * M;
    for (int l = threadIdx.x; l < H; l += blockDim.x) {
        const double x0 = z[slot_of[l]], x1 = z[slot_of[l + H]];
        cddv v;
        if (h == 0) {
            v.re = two_sum(x0, x1);
            v.im = {0.0, 0.0};
        } else {
            ddv d = two_sum(x0, -x1);
            const cddv w = ld4(tw[l]);                 // W^l, W = e^{-2 pi i / M}
            v.re = dmul(d, w.re);
            v.im = dmul(d, w.im);
        }
        A[l] = make_double4(v.re.hi, v.re.lo, v.im.hi, v.im.lo);
    }
    __syncthreads();
    // H-point DIF, twiddle for offset o at half-size hs: W^{o * M / (2 hs)}
    for (int hs = H / 2; hs >= 1; hs >>= 1) {
        for (int b = threadIdx.x; b < H / 2; b += blockDim.x) {
            const int blk = b / hs, o = b % hs;
            const int i0 = blk * 2 * hs + o, i1 = i0 + hs;
            const cddv x = ld4(A[i0]), y = ld4(A[i1]);
            const cddv s = cadd(x, y);
            const cddv d = cmul(csub(x, y), ld4(tw[o * (M / (2 * hs))]));
            A[i0] = make_double4(s.re.hi, s.re.lo, s.im.hi, s.im.lo);
            A[i1] = make_double4(d.re.hi, d.re.lo, d.im.hi, d.im.lo);
        }
        __syncthreads();
    }
    int lg = 0;
    while ((1 << lg) < H) ++lg;
    for (int p = threadIdx.x; p < H; p += blockDim.x) {
        const int kp = (int)(__brev((unsigned)p) >> (32 - lg));
        const int k = 2 * kp + h;                       // frequency index in [0, M)
        const cddv X = ld4(A[p]);
        cddv c = cmul(X, ld4(twist[k]));
        const ddv s = {scale_over_M, 0.0};
        m[(size_t)ct * N + k] = dd_round(dmul(c.re, s));
        m[(size_t)ct * N + k + M] = dd_round(dmul(c.im, s));
    }
}

struct OpSignedRows {
    static const char* family() { return "encode_ntt"; }
    const i64* m;       // [n][N]
    u64* out;           // [n][L][N]
    int n, L, N;
    __host__ __device__ int count() const { return n * L; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int p, int) const { return p % L; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& P) const { return from_signed(m[(size_t)(p / L) * N + j], P); }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC&) const { out[(size_t)p * N + j] = v; }
};

size_t encode_scratch_bytes(const fhe_ctx* c, uint32_t n_ct) { return (size_t)n_ct * c->N * sizeof(i64); }

void encode_coefficients(const fhe_ctx* c, const double* slots, uint32_t n_ct, double scale, i64* m, cudaStream_t st)
{
    const int N = (int)c->N;
    const size_t smem = (size_t)(N / 4) * sizeof(double4);
    static size_t configured = 0;
    if (configured < smem) {
        cudaFuncSetAttribute(k_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = smem;
    }
    int thr = N / 8;
    thr = thr < 32 ? 32 : (thr > 512 ? 512 : thr);
    {
    LaunchScope ls(c, "encode_fft", st);
    k_encode_kernel<<<2 * n_ct, thr, smem, st>>>(slots, c->d_slot_of, c->d_enc_tw, c->d_enc_twist,
                                                 scale / (double)(N / 2), N, m);
    }
}

void k_encode(const fhe_ctx* c, const double* slots, uint32_t n_ct, uint32_t L, double scale, u64* pt, void* scratch,
              cudaStream_t st)
{
    if (n_ct == 0) return;
    i64* m = (i64*)scratch;
    encode_coefficients(c, slots, n_ct, scale, m, st);
    OpSignedRows op{m, pt, (int)n_ct, (int)L, (int)c->N};
    launch_ntt<false>(c, op, st);
}

// ---------------------------------------------------------------- decode
// z_j = Re Z_{l(j)} / scale, Z = DFT_{N/2}(c_k zeta^k) with e^{+2 pi i / M},
// c_k = m_k + i m_{k+N/2}; FP64, one block per ciphertext.
__global__ void __launch_bounds__(512) k_decode_kernel(const i64* __restrict__ m, const uint32_t* __restrict__ slot_of,
                                                        const double4* __restrict__ tw, const double4* __restrict__ twist,
                                                        double inv_scale, int N, double* __restrict__ slots)
{
    extern __shared__ double2 B[];       // N/2 complex doubles
    const int M = N / 2;
    const int ct = blockIdx.x;
    const i64* mc = m + (size_t)ct * N;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        const double a = (double)mc[k], b = (double)mc[k + M];
        const double4 t = twist[k];                     // zeta^{-k}: use its conjugate
        const double wr = t.x, wi = -t.z;
        B[k] = make_double2(a * wr - b * wi, a * wi + b * wr);
    }
    __syncthreads();
    for (int hs = M / 2; hs >= 1; hs >>= 1) {
        for (int b = threadIdx.x; b < M / 2; b += blockDim.x) {
            const int blk = b / hs, o = b % hs;
            const int i0 = blk * 2 * hs + o, i1 = i0 + hs;
            const double2 x = B[i0], y = B[i1];
            const double4 w4 = tw[o * (M / (2 * hs))];  // W^e, W = e^{-2 pi i / M}: conjugate
            const double wr = w4.x, wi = -w4.z;
            const double dr = x.x - y.x, di = x.y - y.y;
            B[i0] = make_double2(x.x + y.x, x.y + y.y);
            B[i1] = make_double2(dr * wr - di * wi, dr * wi + di * wr);
        }
        __syncthreads();
    }
    int lg = 0;
    while ((1 << lg) < M) ++lg;
    for (int l = threadIdx.x; l < M; l += blockDim.x) {
        const int p = (int)(__brev((unsigned)l) >> (32 - lg));
        slots[(size_t)ct * M + slot_of[l]] = B[p].x * inv_scale;
    }
}

void k_decode(const fhe_ctx* c, const i64* m, uint32_t n_ct, double scale, double* slots, cudaStream_t st)
{
    if (n_ct == 0) return;
    const int N = (int)c->N;
    const size_t smem = (size_t)(N / 2) * sizeof(double2);
    static size_t configured = 0;
    if (configured < smem) {
        cudaFuncSetAttribute(k_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = smem;
    }
    int thr = N / 4;
    thr = thr < 32 ? 32 : (thr > 512 ? 512 : thr);
    LaunchScope ls(c, "decode_fft", st);
    k_decode_kernel<<<n_ct, thr, smem, st>>>(m, c->d_slot_of, c->d_enc_tw, c->d_enc_twist, 1.0 / scale, N, slots);
}

}  // namespace fhe
