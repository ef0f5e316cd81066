// k_mac.cu -- multiply-accumulate of dense / convolution layers.
#include "launch.cuh"

namespace fhe {

// Tiled form: rows sharing one column list are computed together, up to
// kMacTile per thread, so each input word is loaded once per tile.
//   tiles[t] = {col_off, K, n_rows, w_off}; rows[t * kMacTile + o] = output row;
//   W[((w_off + e) * L + r) * kMacTile + o] = weight residue of (row o, term e)
// (the tile's weights of one term and residue are contiguous: kMacTile / 2 vector loads).
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
// fewer than 2^20 terms).  S1 is formed Karatsuba-style as
// sum (xL + xH)(wL + wH) - S0 - S2 (limb sums < 2^22, products < 2^44), so a
// term costs three multiply-adds.
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

// NR: rows computed per thread (<= kMacTile); a layer whose tiles hold at most
// five rows (the convolution: five filters over one receptive field) skips
// the sixth row's products
template <int NR>
__global__ void __launch_bounds__(256, 2) k_mac_tiled_kernel(const u64* __restrict__ X, const uint4* __restrict__ tiles,
                                                           const uint32_t* __restrict__ rows,
                                                           const uint32_t* __restrict__ col,
                                                           const u64* __restrict__ W, u64* __restrict__ Y, int L, int N,
                                                           const PrimeC* __restrict__ pc, uint64_t skip_mask)
{
    const uint4 tl = tiles[blockIdx.x];
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    const int kr = blockIdx.z;
    const int r = kr % L;
    if (j >= N || ((skip_mask >> r) & 1u)) return;
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
        // terms four at a time; the next four inputs are loaded before the
        // current four are multiplied (their latency hides behind the MACs)
        u64 xn[4];
        if (K >= 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) xn[u] = Xj[(size_t)__ldg(&cl[u]) * ct_stride];
        }
        for (; e + 4 <= K; e += 4) {
            u64 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = xn[u];
            if (e + 8 <= K) {
#pragma unroll
                for (int u = 0; u < 4; ++u) xn[u] = Xj[(size_t)__ldg(&cl[e + 4 + u]) * ct_stride];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t xl = (uint32_t)(x[u] & kLimbMask), xh = (uint32_t)(x[u] >> 21), xs = xl + xh;
                const ulonglong2* we = w2 + (size_t)(e + u) * wstep;
#pragma unroll
                for (int o2 = 0; o2 < kMacTile / 2; ++o2) {
                    const ulonglong2 wv = __ldg(&we[o2]);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int o = 2 * o2 + h;
                        if (o >= NR) continue;
                        const u64 wd = h ? wv.y : wv.x;
                        const uint32_t wl = (uint32_t)wd, wh = (uint32_t)(wd >> 32);
                        s0[o] += (u64)xl * wl;
                        s1[o] += (u64)xs * (wl + wh);
                        s2[o] += (u64)xh * wh;
                    }
                }
            }
        }
        for (; e < K; ++e) {
            const u64 xv = Xj[(size_t)__ldg(&cl[e]) * ct_stride];
            const uint32_t xl = (uint32_t)(xv & kLimbMask), xh = (uint32_t)(xv >> 21), xs = xl + xh;
            const ulonglong2* we = w2 + (size_t)e * wstep;
#pragma unroll
            for (int o2 = 0; o2 < kMacTile / 2; ++o2) {
                const ulonglong2 wv = __ldg(&we[o2]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int o = 2 * o2 + h;
                    if (o >= NR) continue;
                    const u64 wd = h ? wv.y : wv.x;
                    const uint32_t wl = (uint32_t)wd, wh = (uint32_t)(wd >> 32);
                    s0[o] += (u64)xl * wl;
                    s1[o] += (u64)xs * (wl + wh);
                    s2[o] += (u64)xh * wh;
                }
            }
        }
#pragma unroll
        for (int o = 0; o < NR; ++o)
            if (o < (int)tl.z)
                Y[(size_t)rows[blockIdx.x * kMacTile + o] * ct_stride + off] =
                    limb_combine(s0[o], s1[o] - s0[o] - s2[o], s2[o], P);
        return;
    }
    u64 lo[kMacTile], hi[kMacTile];
#pragma unroll
    for (int o = 0; o < kMacTile; ++o) lo[o] = hi[o] = 0;
    uint32_t e = 0;
    int cnt = 0;
    // products are below q^2, so a high word is below 2^58 for q < 2^61 and
    // below 2^60 for q < 2^62: fold before 32 (resp. 16) high words can overflow
    const int fold = P.q < (1ull << 61) ? 32 : 16;
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
                if (2 * o2 + 1 < NR) mac128(lo[2 * o2 + 1], hi[2 * o2 + 1], x[u], wv.y);
            }
        }
        cnt += 4;
        if (cnt == fold) {
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
            if (2 * o2 + 1 < NR) mac128(lo[2 * o2 + 1], hi[2 * o2 + 1], x, wv.y);
        }
    }
#pragma unroll
    for (int o = 0; o < NR; ++o)
        if (o < (int)tl.z) Y[(size_t)rows[blockIdx.x * kMacTile + o] * ct_stride + off] = reduce128(hi[o], lo[o], P);
}

void k_linear_mac_tiled(const fhe_ctx* c, const u64* X, const uint4* tiles, uint32_t n_tiles, const uint32_t* rows,
                        const uint32_t* col, const u64* W, uint32_t L, u64* Y, cudaStream_t st, uint64_t skip_mask,
                        uint32_t max_tile_rows)
{
    if (n_tiles == 0 || (L < 64 && (skip_mask & ((1ull << L) - 1)) == (1ull << L) - 1)) return;
    const int N = (int)c->N;
    const int tpb = N < 256 ? N : 256;
    dim3 grid(n_tiles, (N + tpb - 1) / tpb, 2 * L);
    LaunchScope ls(c, "mac", st);
    if (max_tile_rows <= 5)
        k_mac_tiled_kernel<5><<<grid, tpb, 0, st>>>(X, tiles, rows, col, W, Y, (int)L, N, c->d_pc, skip_mask);
    else
        k_mac_tiled_kernel<kMacTile><<<grid, tpb, 0, st>>>(X, tiles, rows, col, W, Y, (int)L, N, c->d_pc, skip_mask);
}


}  // namespace fhe
