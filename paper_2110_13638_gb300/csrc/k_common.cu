// k_common.cu -- launch accounting, plain transforms, element-wise kernels,
// per-level division constants.
#include <map>
#include <mutex>

#include "launch.cuh"

namespace fhe {

static std::atomic<uint64_t> g_launches{0};

uint64_t launch_count() { return g_launches.load(); }

LaunchScope::LaunchScope(const fhe_ctx* ctx, const char* family, cudaStream_t s) : c(ctx), st(s)
{
    g_launches.fetch_add(1);
    if (c && !c->prof_family.empty() && c->prof_family == family) {
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

void ensure_smem(const void* kernel, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    size_t& have = done[{kernel, dev}];
    if (have < bytes) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        have = bytes;
    }
}

const char* ntt_variant_name(int v)
{
    switch (v) {
    case 1: return "one block per transform, radix-8 passes, 1024 threads";
    case 2: return "two-pass column/row tiles, radix-16";
    case 3: return "two-pass column/row tiles, radix-8";
    case 4: return "one block per transform, radix-8, loads and stores fused into the first and last pass";
    case 5: return "one block per transform, radix-16, loads and stores fused into the first and last pass";
    case 6: return "key-switching digit transforms split over two blocks (one per output half), radix-16";
    case 7: return "key-switching digit transforms on a cluster of four blocks (one per coefficient quarter), "
                   "accumulators in shared memory";
    case 8: return "one block of N/32 threads per transform: the first log2 N - 10 stages block-wide, then each "
                   "warp runs a 1024-point sub-transform, 32 values per lane (one block barrier per transform)";
    default: return "one block per transform, radix-16 passes, 512 threads";
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
        const uint32_t r = (uint32_t)(i >> logN) % (uint32_t)L;      // row index math in 32 bits
        const u64 q = pc[r].q;
        out[i] = add_mod(a[i], b[i], q);
    }
}


void k_add(const fhe_ctx* c, const u64* a, const u64* b, u64* out, uint32_t n_ct, uint32_t comps, uint32_t L,
           cudaStream_t st)
{
    size_t total = (size_t)n_ct * comps * L * c->N;
    if (!total) return;
    LaunchScope ls(c, "elementwise", st);
    k_add_kernel<<<ew_grid(total), 256, 0, st>>>(a, b, out, total, (int)L, (int)c->logN, c->d_pc);
}

// thread covers (ct, r, j); a squaring (a == b) needs three products
template <bool SQUARE>
__global__ void k_tensor_kernel(const u64* __restrict__ a, const u64* __restrict__ b, u64* __restrict__ out,
                                size_t total, int L, int logN, const PrimeC* __restrict__ pc)
{
    const size_t per_comp = (size_t)L << logN;
    const size_t Nm = ((size_t)1 << logN) - 1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t row = (uint32_t)(i >> logN);          // ct * L + r, 32-bit index math
        const uint32_t ct = row / (uint32_t)L, r = row - ct * (uint32_t)L;
        const size_t w = ((size_t)r << logN) + (i & Nm);
        const PrimeC P = pc[r];
        const u64* A = a + (size_t)ct * 2 * per_comp;
        u64* O = out + (size_t)ct * 3 * per_comp;
        const u64 a0 = A[w], a1 = A[per_comp + w];
        if constexpr (SQUARE) {
            const u64 m = mul_mod_r(a0, a1, P);
            O[w] = mul_mod_r(a0, a0, P);
            O[per_comp + w] = add_mod(m, m, P.q);
            O[2 * per_comp + w] = mul_mod_r(a1, a1, P);
        } else {
            const u64* B = b + (size_t)ct * 2 * per_comp;
            const u64 b0 = B[w], b1 = B[per_comp + w];
            O[w] = mul_mod_r(a0, b0, P);
            O[per_comp + w] = add_mod(mul_mod_r(a0, b1, P), mul_mod_r(a1, b0, P), P.q);
            O[2 * per_comp + w] = mul_mod_r(a1, b1, P);
        }
    }
}

void k_tensor(const fhe_ctx* c, const u64* a, const u64* b, u64* out3, uint32_t n_ct, uint32_t L, cudaStream_t st)
{
    const size_t total = (size_t)n_ct * L * c->N;
    if (!total) return;
    LaunchScope ls(c, "tensor", st);
    if (a == b)
        k_tensor_kernel<true><<<ew_grid(total), 256, 0, st>>>(a, b, out3, total, (int)L, (int)c->logN, c->d_pc);
    else
        k_tensor_kernel<false><<<ew_grid(total), 256, 0, st>>>(a, b, out3, total, (int)L, (int)c->logN, c->d_pc);
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
        const uint32_t row = (uint32_t)(i >> logN);          // (ct, comp, r) with r < L_out
        const uint32_t poly = row / (uint32_t)L_out, r = row - poly * (uint32_t)L_out;
        const uint32_t ct = poly / (uint32_t)comps;
        const PrimeC P = pc[r];
        const u64 x = in[(((size_t)poly * L_in + r) << logN) + (i & Nm)];
        out[i] = mul_mod_r(x, cres[(size_t)ct * cstride + r], P);
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
        const uint32_t row = (uint32_t)(i >> logN);          // (ct, r) over comp 0 only
        const uint32_t n = row / (uint32_t)L, r = row - n * (uint32_t)L;
        const size_t idx = (((size_t)n * 2 * L + r) << logN) + (i & (((size_t)1 << logN) - 1));
        ct[idx] = add_mod(ct[idx], cres[(size_t)n * cstride + r], pc[r].q);
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
                                      const u64* __restrict__ c1, const PrimeC* __restrict__ pc, bool accumulate)
{
    const size_t Nm = ((size_t)1 << logN) - 1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t row = (uint32_t)(i >> logN);          // (ct, comp, r), r < L1
        const uint32_t poly = row / (uint32_t)L1, r = row - poly * (uint32_t)L1;
        const PrimeC P = pc[r];
        const u64 xv = x[(((size_t)poly * Lx + r) << logN) + (i & Nm)];
        u64 a = mul_mod_r(x2[i], c2[r], P);
        if (accumulate) a = add_mod(t1[i], a, P.q);
        t1[i] = add_mod(a, mul_mod_r(xv, c1[r], P), P.q);
    }
}

void k_poly_combine(const fhe_ctx* c, u64* t1, const u64* x2, const u64* x, uint32_t n_ct, uint32_t L1, uint32_t Lx,
                    const u64* c2, const u64* c1, cudaStream_t st, bool accumulate)
{
    const size_t total = (size_t)n_ct * 2 * L1 * c->N;
    if (!total) return;
    LaunchScope ls(c, "elementwise", st);
    k_poly_combine_kernel<<<ew_grid(total), 256, 0, st>>>(t1, x2, x, total, (int)L1, (int)Lx, (int)c->logN, c2, c1,
                                                          c->d_pc, accumulate);
}

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

// ---------------------------------------------------------------- packed convolution
__global__ void k_plain_mac_kernel(u64* __restrict__ Y, const u64* __restrict__ X, const u64* __restrict__ PT,
                                   size_t total, int F, int n, int L, int p, int k2, int logN,
                                   const PrimeC* __restrict__ pc, bool accumulate)
{
    const size_t Nm = ((size_t)1 << logN) - 1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t row = (uint32_t)(i >> logN);          // ((f * n + ct) * 2 + comp) * L + r
        const uint32_t fc = row / (uint32_t)L, r = row - fc * (uint32_t)L;
        const int comp = (int)(fc & 1);
        const uint32_t fi = fc >> 1;
        const int f = (int)(fi / (uint32_t)n), ct = (int)(fi - (uint32_t)f * (uint32_t)n);
        const int j = (int)(i & Nm);
        const PrimeC P = pc[r];
        const u64 x = X[((((size_t)ct * 2 + comp) * L + r) << logN) + j];
        const u64 w = PT[((((size_t)f * k2 + p) * L + r) << logN) + j];
        u64 v = mul_mod_r(x, w, P);
        if (accumulate) v = add_mod(Y[i], v, P.q);
        Y[i] = v;
    }
}

void k_plain_mac(const fhe_ctx* c, u64* Y, const u64* X, const u64* PT, uint32_t F, uint32_t n, uint32_t L,
                 uint32_t p, uint32_t k2, bool accumulate, cudaStream_t st)
{
    const size_t total = (size_t)F * n * 2 * L * c->N;
    if (!total) return;
    LaunchScope ls(c, "elementwise", st);
    k_plain_mac_kernel<<<ew_grid(total), 256, 0, st>>>(Y, X, PT, total, (int)F, (int)n, (int)L, (int)p, (int)k2,
                                                       (int)c->logN, c->d_pc, accumulate);
}

__global__ void k_add_plain_kernel(u64* __restrict__ out, const u64* __restrict__ bias, size_t total, int n, int L1,
                                   int logN, const PrimeC* __restrict__ pc)
{
    const size_t Nm = ((size_t)1 << logN) - 1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t row = (uint32_t)(i >> logN);          // (f * n + ct) * L1 + r, component 0 only
        const uint32_t fi = row / (uint32_t)L1, r = row - fi * (uint32_t)L1;
        const int f = (int)(fi / (uint32_t)n);
        const size_t o = ((((size_t)fi * 2) * L1 + r) << logN) + (i & Nm);
        out[o] = add_mod(out[o], bias[(((size_t)f * L1 + r) << logN) + (i & Nm)], pc[r].q);
    }
}

void k_add_plain(const fhe_ctx* c, u64* out, const u64* bias, uint32_t F, uint32_t n, uint32_t L1, cudaStream_t st)
{
    const size_t total = (size_t)F * n * L1 * c->N;
    if (!total) return;
    LaunchScope ls(c, "elementwise", st);
    k_add_plain_kernel<<<ew_grid(total), 256, 0, st>>>(out, bias, total, (int)n, (int)L1, (int)c->logN, c->d_pc);
}

__global__ void k_gather_slots_kernel(const double* __restrict__ src, const int64_t* __restrict__ index, size_t total,
                                      double* __restrict__ dst)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int64_t k = index[i];
        dst[i] = k >= 0 ? src[k] : 0.0;
    }
}

void k_gather_slots(const double* src, const int64_t* index, size_t total, double* dst, cudaStream_t st)
{
    if (!total) return;
    LaunchScope ls(nullptr, "gather", st);
    k_gather_slots_kernel<<<ew_grid(total), 256, 0, st>>>(src, index, total, dst);
}

}  // namespace fhe
