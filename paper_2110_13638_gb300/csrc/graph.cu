// graph.cu -- graph objects and encrypted graph evaluation.
//
// Traversal follows Alg. firing / signal_carrier of arXiv 2110.13638 (Sec. 3):
// each input node is stimulated in turn; a node fires once every in-edge
// carries a signal (its inputs stacked in edge order, or summed for ADD);
// its output is set on every out-edge, then each successor is visited.
// Receptors (apply_signal) are the block schedules below; each is a fixed
// sequence of batched kernel launches on the caller's stream:
//   LINEAR  y_o = rescale(sum_e llround(w_e q_{L-1}) x_{col_e}) + llround(b_o s_y)
//   SQUARE  rescale(relin(x (x) x))
//   POLY    degree 3: x2 = rescale(relin(x (x) x));  w = rescale(x * llround(a3 s3));
//           T = relin(x2 (x) w) + x2 * llround(a2 s_2) + drop(x) * llround(a1 q');
//           y = rescale(T) + llround(a0 s_y)
//           (s3 = q' q / s2, s_2 = s q' / s2, s2 = s s / q; q = q_{L-1}, q' = q_{L-2})
//           degree 2: the same without w and the relin(x2 (x) w) term
//           degree 1: y = rescale(x * llround(a1 q)) + llround(a0 s_y)
//   RELU    Eq. relu_approximate with range q: the degree-2 POLY with
//           a0 = q / (3 pi), a1 = 1/2, a2 = 4 / (3 pi q)
// Nominal scales are FP64 values updated in exactly this order.
// A dry run with the same allocation sequence sizes the workspace first.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/fhe.h"
#include "ctx.h"
#include "host_math.h"

using namespace fhe;

namespace {

constexpr uint32_t kMaxPolyDegree = 31;

// Degree > 3: plan of the powers x^i (levels and nominal scales, FP64 in the
// order the receptor computes them) and the combining constants.
struct PowPlan {
    std::vector<uint32_t> j;        // x^i = x^j x^(i - j)
    std::vector<uint32_t> lev;      // level of x^i (lev[1] = L)
    std::vector<double> sc;         // nominal scale of x^i
    uint32_t lstar = 0;             // lowest level among the powers
    std::vector<int64_t> C;         // C[i] = llround(a_i S / s_i) (0 where a_i = 0), C[0] = llround(a_0 s_y)
    double s_T = 0.0, s_y = 0.0;    // scale of the sum (first term's) and of the result
    bool scales_agree = true;
};

struct Sig {
    u64* p = nullptr;
    uint32_t n = 0, L = 0;
    double scale = 0.0;
    bool set = false;
};

static u64 mod_signed(int64_t v, u64 q)
{
    if (v >= 0) return (u64)v % q;
    u64 r = (u64)(-(v + 1)) % q;
    r = (r + 1) % q;
    return r == 0 ? 0 : q - r;
}

static size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

// FHE_MAC_TC=0 keeps dense layers on the integer-pipe MAC (for comparisons)
static bool mac_tc_enabled()
{
    const char* e = std::getenv("FHE_MAC_TC");
    return !(e && e[0] == '0');
}

// balanced base-256 limbs of a centred residue (|v| < 2^40 with five limbs,
// < 2^60 with eight): n - 1 digits in [-128, 127] and a top digit taking the
// rest (the split the tensor-core MAC makes on the device)
static void mac_tc_limbs(int64_t v, int n, int32_t (&d)[8])
{
    int64_t bias = 0;
    for (int a = 0; a + 1 < n; ++a) bias += (int64_t)128 << (8 * a);
    const int64_t u = v + bias;
    const int64_t span = (int64_t)1 << (8 * (n - 1));
    const int64_t low = u & (span - 1);
    for (int a = 0; a + 1 < n; ++a) d[a] = (int32_t)((low >> (8 * a)) & 255) - 128;
    d[n - 1] = (int32_t)((u - low) / span);
}

// bf16 bit pattern of a small integer (|v| <= 256: exact)
static uint16_t bf16_of_small(int32_t v)
{
    const float f = (float)v;
    uint32_t bits;
    std::memcpy(&bits, &f, 4);
    return (uint16_t)(bits >> 16);
}

struct Exec {
    fhe_ctx* c;
    fhe_graph* g;
    cudaStream_t st;
    bool dry;
    Arena ar;
    size_t need = 0;
    int rc = FHE_OK;
    std::vector<Sig> edge;
    std::vector<char> fired;
    std::vector<Sig> outputs;            // per node (OUTPUT nodes only)
    std::vector<std::vector<uint32_t>> in_e, out_e;

    void* take(size_t bytes)
    {
        if (dry) {
            need += al(bytes);
            return nullptr;
        }
        void* p = ar.take(bytes);
        if (!p && rc == FHE_OK) rc = fail(FHE_ENOMEM, "graph workspace exhausted");
        return p;
    }
    size_t cts(uint32_t n, uint32_t comps, uint32_t L) const { return (size_t)n * comps * L * c->N * 8; }
    bool ok() const { return rc == FHE_OK; }
    int err(int code, const char* m)
    {
        if (rc == FHE_OK) rc = fail(code, m);
        return rc;
    }

    // ------------------------------------------------ constants cache
    fhe_node_const* node_const(uint32_t i, uint32_t L, double s_in)
    {
        fhe_node_const& nc = g->cache[i];
        const bool tc_on = mac_tc_enabled();
        if (nc.buf && nc.L == L && nc.s_in == s_in && nc.tc_on == tc_on) return &nc;
        if (nc.buf) {
            cudaStreamSynchronize(st);
            cudaFree(nc.buf);
            nc = fhe_node_const();
        }
        const fhe_graph_node& nd = g->nodes[i];
        if (nd.kind == FHE_NODE_CONV_PACKED) return conv_const(i, L, s_in);
        std::vector<char> host;
        auto put = [&](const void* src, size_t bytes) {
            size_t off = host.size();
            host.resize(off + al(bytes));
            std::memcpy(host.data() + off, src, bytes);
            return off;
        };
        size_t o_rp = 0, o_tr = 0, o_col = 0, o_W = 0, o_b = 0, o_c3 = 0, o_c2 = 0, o_c1 = 0, o_c0 = 0;
        size_t o_c3s = 0, o_c2s = 0, o_c1s = 0;
        size_t o_tcW[2] = {0, 0}, o_tcr[2] = {0, 0};
        uint32_t tc_tiles[2] = {0, 0}, tc_K = 0;
        uint64_t tc_mask[2] = {0, 0};
        if (nd.kind == FHE_NODE_LINEAR) {
            const double qd = (double)c->primes[L - 1];
            // group rows with identical column lists, split groups into tiles
            std::map<std::vector<uint32_t>, std::vector<uint32_t>> groups;
            std::vector<std::vector<uint32_t>> order;
            for (uint32_t o = 0; o < nd.n_out; ++o) {
                std::vector<uint32_t> cols(nd.col_idx.begin() + nd.row_ptr[o], nd.col_idx.begin() + nd.row_ptr[o + 1]);
                auto it = groups.find(cols);
                if (it == groups.end()) {
                    groups[cols] = {o};
                    order.push_back(cols);
                } else {
                    it->second.push_back(o);
                }
            }
            std::vector<uint4> tiles;
            std::vector<uint32_t> trows, tcol;
            std::vector<u64> W;
            for (const auto& cols : order) {
                const std::vector<uint32_t>& rs = groups[cols];
                const uint32_t col_off = (uint32_t)tcol.size();
                tcol.insert(tcol.end(), cols.begin(), cols.end());
                for (size_t t0 = 0; t0 < rs.size(); t0 += kMacTile) {
                    const uint32_t nr = (uint32_t)std::min<size_t>(kMacTile, rs.size() - t0);
                    const uint32_t w_off = (uint32_t)(W.size() / ((size_t)L * kMacTile));  // in terms
                    tiles.push_back(make_uint4(col_off, (uint32_t)cols.size(), nr, w_off));
                    for (int o = 0; o < kMacTile; ++o) trows.push_back(o < (int)nr ? rs[t0 + o] : 0u);
                    W.resize(W.size() + (size_t)cols.size() * kMacTile * L, 0);
                    for (size_t e = 0; e < cols.size(); ++e)
                        for (uint32_t o = 0; o < nr; ++o) {
                            const uint32_t row = rs[t0 + o];
                            const double wv = nd.weight[nd.row_ptr[row] + e];
                            const int64_t w = (int64_t)std::llround(wv * qd);
                            for (uint32_t r = 0; r < L; ++r) {
                                u64 wr = mod_signed(w, c->primes[r]);
                                if (c->primes[r] < kLimbPrimeBound)          // 21-bit limbs for the limb MAC
                                    wr = (wr & ((1ull << 21) - 1)) | ((wr >> 21) << 32);
                                W[(((size_t)w_off + e) * L + r) * kMacTile + o] = wr;
                            }
                        }
                }
            }
            const double s_out = (s_in * qd) / qd;
            std::vector<u64> B((size_t)nd.n_out * (L - 1));
            for (uint32_t o = 0; o < nd.n_out; ++o) {
                const int64_t b = (int64_t)std::llround(nd.bias[o] * s_out);
                for (uint32_t r = 0; r + 1 < L; ++r) B[(size_t)o * (L - 1) + r] = mod_signed(b, c->primes[r]);
            }
            // dense layer (one column list shared by every row): its residues go
            // to the tensor-core MAC as bf16 limb tiles, five limbs for primes
            // below 2^41 and eight below 2^61 (at most 8192 terms: the 64-bit
            // class sums of the epilogue stay exact)
            const bool dense = order.size() == 1 && order[0].size() >= (size_t)kMacTcChunk &&
                               order[0].size() <= 8192 && nd.n_out >= 16 && c->N % 128 == 0 && 2 * L <= 64;
            if (tc_on && dense)
                for (uint32_t r = 0; r < L; ++r) {
                    if (c->primes[r] < kMacTcPrimeBound5) tc_mask[0] |= 1ull << r;
                    else if (c->primes[r] < kMacTcPrimeBound8) tc_mask[1] |= 1ull << r;
                }
            for (int part = 0; part < 2; ++part) {
                if (!tc_mask[part]) continue;
                const int limbs = part == 0 ? 5 : 8;
                const size_t NT = part == 0 ? kMacTcRows : kMacTcRows8;
                const std::vector<uint32_t>& cols = order[0];
                const std::vector<uint32_t>& rs = groups[cols];
                tc_K = (uint32_t)cols.size();
                tc_tiles[part] = (uint32_t)((rs.size() + NT - 1) / NT);
                const size_t n_chunks = (tc_K + kMacTcChunk - 1) / kMacTcChunk;
                const size_t plane = NT * kMacTcChunk;
                const size_t n_res = (size_t)__builtin_popcountll(tc_mask[part]);
                std::vector<uint16_t> Wl(n_res * tc_tiles[part] * n_chunks * limbs * plane, 0);
                std::vector<uint32_t> trow((size_t)tc_tiles[part] * NT, 0xFFFFFFFFu);
                for (size_t idx = 0; idx < rs.size(); ++idx) trow[idx] = rs[idx];
                size_t ri = 0;
                for (uint32_t r = 0; r < L; ++r) {
                    if (!((tc_mask[part] >> r) & 1u)) continue;
                    const u64 q = c->primes[r], half = (q - 1) / 2;
                    for (size_t idx = 0; idx < rs.size(); ++idx) {
                        const size_t t = idx / NT, o = idx % NT;
                        const uint32_t row = rs[idx];
                        for (uint32_t e = 0; e < tc_K; ++e) {
                            const int64_t w = (int64_t)std::llround(nd.weight[nd.row_ptr[row] + e] * qd);
                            const u64 wr = mod_signed(w, q);
                            const int64_t wc = wr > half ? (int64_t)wr - (int64_t)q : (int64_t)wr;
                            int32_t d[8];
                            mac_tc_limbs(wc, limbs, d);
                            const size_t ch = e / kMacTcChunk, k = e % kMacTcChunk;
                            const size_t pos = ((o >> 3) * (kMacTcChunk / 8) + (k >> 3)) * 64 + (o & 7) * 8 + (k & 7);
                            for (int b = 0; b < limbs; ++b)
                                Wl[(((ri * tc_tiles[part] + t) * n_chunks + ch) * limbs + b) * plane + pos] =
                                    bf16_of_small(d[b]);
                        }
                    }
                    ++ri;
                }
                o_tcW[part] = put(Wl.data(), Wl.size() * 2);
                o_tcr[part] = put(trow.data(), trow.size() * 4);
            }
            nc.n_tiles = (uint32_t)tiles.size();
            nc.max_tile_rows = 0;
            for (const uint4& tl : tiles) nc.max_tile_rows = std::max(nc.max_tile_rows, tl.z);
            o_rp = put(tiles.data(), std::max<size_t>(1, tiles.size()) * sizeof(uint4));
            o_tr = put(trows.data(), std::max<size_t>(1, trows.size()) * 4);
            o_col = put(tcol.data(), std::max<size_t>(1, tcol.size()) * 4);
            o_W = put(W.data(), std::max<size_t>(1, W.size()) * 8);
            o_b = put(B.data(), std::max<size_t>(1, B.size()) * 8);
        } else if (nd.kind == FHE_NODE_POLY && nd.degree > 3) {
            const PowPlan P = pow_plan(nd, L, s_in);
            const uint32_t ls = P.lstar;
            std::vector<u64> cr((size_t)(nd.degree + 1) * ls, 0);
            for (uint32_t k = 1; k <= nd.degree; ++k)
                for (uint32_t r = 0; r < ls; ++r) cr[(size_t)(k - 1) * ls + r] = mod_signed(P.C[k], c->primes[r]);
            for (uint32_t r = 0; r + 1 < ls; ++r) cr[(size_t)nd.degree * ls + r] = mod_signed(P.C[0], c->primes[r]);
            o_c0 = put(cr.data(), cr.size() * 8);
        } else if (nd.kind == FHE_NODE_POLY || nd.kind == FHE_NODE_RELU) {
            PolyK k = poly_constants(nd, L, s_in);
            std::vector<u64> r3(L), r2(L), r1(L), r0(L);          // residues of C3..C0 at every prime of level L
            for (uint32_t r = 0; r < L; ++r) {
                r3[r] = mod_signed(k.C3, c->primes[r]);
                r2[r] = mod_signed(k.C2, c->primes[r]);
                r1[r] = mod_signed(k.C1, c->primes[r]);
                r0[r] = mod_signed(k.C0, c->primes[r]);
            }
            std::vector<u64> r3s(L), r2s(L), r1s(L);              // Shoup quotients of C3..C1
            for (uint32_t r = 0; r < L; ++r) {
                r3s[r] = shoup(r3[r], c->primes[r]);
                r2s[r] = shoup(r2[r], c->primes[r]);
                r1s[r] = shoup(r1[r], c->primes[r]);
            }
            o_c3 = put(r3.data(), r3.size() * 8);
            o_c2 = put(r2.data(), r2.size() * 8);
            o_c1 = put(r1.data(), r1.size() * 8);
            o_c0 = put(r0.data(), r0.size() * 8);
            o_c3s = put(r3s.data(), r3s.size() * 8);
            o_c2s = put(r2s.data(), r2s.size() * 8);
            o_c1s = put(r1s.data(), r1s.size() * 8);
        } else {
            return nullptr;
        }
        cudaError_t e = cudaMalloc(&nc.buf, host.size());
        if (e == cudaSuccess) e = cudaMemcpy(nc.buf, host.data(), host.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = cuda_check(e, "graph constants");
            return nullptr;
        }
        char* b = (char*)nc.buf;
        nc.L = L;
        nc.s_in = s_in;
        nc.tc_on = tc_on;
        if (nd.kind == FHE_NODE_LINEAR) {
            for (int part = 0; part < 2; ++part) {
                if (!tc_mask[part]) continue;
                nc.tc[part].W = (uint16_t*)(b + o_tcW[part]);
                nc.tc[part].rows = (uint32_t*)(b + o_tcr[part]);
                nc.tc[part].tiles = tc_tiles[part];
                nc.tc[part].mask = tc_mask[part];
            }
            nc.tc_K = tc_K;
            nc.tiles = (uint4*)(b + o_rp);
            nc.tile_rows = (uint32_t*)(b + o_tr);
            nc.col = (uint32_t*)(b + o_col);
            nc.W = (u64*)(b + o_W);
            nc.bias = (u64*)(b + o_b);
        } else if (nd.kind == FHE_NODE_POLY && nd.degree > 3) {
            nc.cpow = (u64*)(b + o_c0);
        } else {
            nc.c3 = (u64*)(b + o_c3);
            nc.c2 = (u64*)(b + o_c2);
            nc.c1 = (u64*)(b + o_c1);
            nc.c0 = (u64*)(b + o_c0);
            nc.c3s = (u64*)(b + o_c3s);
            nc.c2s = (u64*)(b + o_c2s);
            nc.c1s = (u64*)(b + o_c1s);
        }
        return &nc;
    }

    // ------------------------------------------------ packed convolution
    // output slots b S + s r W + s c of every image b, row r, column c
    std::vector<uint32_t> conv_valid(const fhe_graph_node& nd) const
    {
        const uint32_t H = nd.conv[0], W = nd.conv[1], k = nd.conv[2], st_ = nd.conv[3], imgs = nd.conv[4],
                       S = nd.conv[5];
        const uint32_t OH = (H - k) / st_ + 1, OW = (W - k) / st_ + 1;
        std::vector<uint32_t> v;
        for (uint32_t b = 0; b < imgs; ++b)
            for (uint32_t r = 0; r < OH; ++r)
                for (uint32_t cc = 0; cc < OW; ++cc) v.push_back(b * S + st_ * r * W + st_ * cc);
        return v;
    }

    // mask-and-kernel plaintexts (scale q_{L-1}, level L) and bias plaintexts
    // (scale of the output, level L-1), encoded on the device once per level
    fhe_node_const* conv_const(uint32_t i, uint32_t L, double s_in)
    {
        fhe_node_const& nc = g->cache[i];
        const fhe_graph_node& nd = g->nodes[i];
        const size_t N = c->N, M = N / 2;
        const uint32_t F = nd.n_out, k2 = nd.conv[2] * nd.conv[2];
        const std::vector<uint32_t> valid = conv_valid(nd);
        for (uint32_t v : valid)
            if (v >= M) { err(FHE_EINVAL, "packed images exceed the ciphertext's slots"); return nullptr; }
        const double qd = (double)c->primes[L - 1];
        const double s_out = (s_in * qd) / qd;
        std::vector<double> V((size_t)(F * k2 + F) * M, 0.0);
        for (uint32_t f = 0; f < F; ++f) {
            for (uint32_t p = 0; p < k2; ++p)
                for (uint32_t v : valid) V[((size_t)f * k2 + p) * M + v] = nd.weight[(size_t)f * k2 + p];
            for (uint32_t v : valid) V[((size_t)F * k2 + f) * M + v] = nd.bias[f];
        }
        const size_t b_pt = al((size_t)F * k2 * L * N * 8), b_bias = al((size_t)F * (L - 1) * N * 8);
        const size_t b_v = al(V.size() * 8), b_s = al(encode_scratch_bytes(c, F * k2));
        char* tmp = nullptr;
        cudaError_t e = cudaMalloc(&nc.buf, b_pt + b_bias);
        if (e == cudaSuccess) e = cudaMalloc((void**)&tmp, b_v + b_s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, V.data(), V.size() * 8, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(tmp);
            rc = cuda_check(e, "packed convolution constants");
            return nullptr;
        }
        nc.pt = (u64*)nc.buf;
        nc.bias_pt = (u64*)((char*)nc.buf + b_pt);
        k_encode(c, (const double*)tmp, F * k2, L, qd, nc.pt, tmp + b_v, st);
        k_encode(c, (const double*)tmp + (size_t)F * k2 * M, F, L - 1, s_out, nc.bias_pt, tmp + b_v, st);
        e = cudaStreamSynchronize(st);
        cudaFree(tmp);
        if (e != cudaSuccess) { rc = cuda_check(e, "packed convolution constants"); return nullptr; }
        nc.L = L;
        nc.s_in = s_in;
        return &nc;
    }

    Sig conv_packed(uint32_t i, const Sig& x)
    {
        Sig y;
        const fhe_graph_node& nd = g->nodes[i];
        const uint32_t L = x.L, n = x.n, F = nd.n_out, k = nd.conv[2], W = nd.conv[1];
        if (L < 2) { err(FHE_ELEVEL, "packed convolution needs two primes"); return y; }
        u64* R = (u64*)take(cts(n, 2, L));
        u64* d3 = (u64*)take(cts(n, 3, L));
        void* rs = take(relin_scratch_bytes(c, n, L));
        u64* Y = (u64*)take(cts(F * n, 2, L));
        void* ss = take(rescale_scratch_bytes(c, F * n, 2));
        u64* out = (u64*)take(cts(F * n, 2, L - 1));
        if (!dry && ok()) {
            fhe_ctx* root = c->parent ? c->parent : c;
            std::vector<int64_t> offs;
            for (uint32_t dr = 0; dr < k; ++dr)
                for (uint32_t dc = 0; dc < k; ++dc) offs.push_back((int64_t)(dr * W + dc));
            rc = galois_keys_for(root, offs, st);
            if (!ok()) return y;
            fhe_node_const* kc = node_const(i, L, x.scale);
            if (!kc) return y;
            for (uint32_t p = 0; p < k * k; ++p) {
                const u64* src = x.p;
                if (offs[p] != 0) {
                    const u64 gk = galois_element_of(c, offs[p]);
                    k_automorph(c, x.p, d3, n, L, gk, st);
                    k_relin(c, d3, R, n, L, rs, st, root->galois[gk]);
                    src = R;
                }
                k_plain_mac(c, Y, src, kc->pt, F, n, L, p, k * k, p > 0, st);
            }
            k_rescale(c, Y, out, F * n, 2, L, nullptr, 0, ss, st);
            k_add_plain(c, out, kc->bias_pt, F, n, L - 1, st);
        }
        const double qd = (double)c->primes[L - 1];
        y.p = out;
        y.n = F * n;
        y.L = L - 1;
        y.scale = (x.scale * qd) / qd;
        y.set = true;
        return y;
    }

    // ------------------------------------------------ polynomials of degree > 3
    PowPlan pow_plan(const fhe_graph_node& nd, uint32_t L, double s) const
    {
        const uint32_t d = nd.degree;
        PowPlan p;
        p.j.assign(d + 1, 0);
        p.lev.assign(d + 1, 0);
        p.sc.assign(d + 1, 0.0);
        p.C.assign(d + 1, 0);
        p.lev[1] = L;
        p.sc[1] = s;
        p.lstar = L;
        for (uint32_t i = 2; i <= d; ++i) {
            uint32_t j = 1;
            while ((j << 1) <= i) j <<= 1;
            if (j == i) j = i / 2;
            const uint32_t lv = std::min(p.lev[j], p.lev[i - j]);
            if (lv < 2) return p;                         // lstar stays > 0: caller reports
            p.j[i] = j;
            p.lev[i] = lv - 1;
            p.sc[i] = (p.sc[j] * p.sc[i - j]) / (double)c->primes[lv - 1];
            p.lstar = std::min(p.lstar, p.lev[i]);
        }
        if (p.lstar < 2) return p;
        const double S = s * (double)c->primes[p.lstar - 1];
        bool first = true;
        for (uint32_t i = 1; i <= d; ++i) {
            if (nd.poly[i] == 0.0) continue;
            const double sig = S / p.sc[i];
            p.C[i] = (int64_t)std::llround(nd.poly[i] * sig);
            const double st_i = p.sc[i] * sig;
            if (first) p.s_T = st_i;
            else p.scales_agree &= scale_match(p.s_T, st_i);
            first = false;
        }
        p.s_y = p.s_T / (double)c->primes[p.lstar - 1];
        p.C[0] = (int64_t)std::llround(nd.poly[0] * p.s_y);
        return p;
    }

    Sig poly_powers(uint32_t i, const Sig& x)
    {
        Sig y;
        const fhe_graph_node& nd = g->nodes[i];
        const uint32_t d = nd.degree, n = x.n;
        const PowPlan P = pow_plan(nd, x.L, x.scale);
        for (uint32_t k = 2; k <= d; ++k)
            if (P.lev[k] == 0) { err(FHE_ELEVEL, "not enough primes for this polynomial degree"); return y; }
        if (P.lstar < 2) { err(FHE_ELEVEL, "not enough primes for this polynomial degree"); return y; }
        if (!P.scales_agree) { err(FHE_ESCALE, "polynomial terms disagree in scale"); return y; }
        std::vector<Sig> pw(d + 1);
        pw[1] = x;
        for (uint32_t k = 2; k <= d; ++k) {
            const uint32_t j = P.j[k], lv = P.lev[k] + 1;
            const Sig A = drop_to(pw[j], lv), B = (j == k - j) ? A : drop_to(pw[k - j], lv);
            u64* T3 = (u64*)take(cts(n, 3, lv));
            void* rs = take(relin_rescale_scratch_bytes(c, n, lv));
            u64* out = (u64*)take(cts(n, 2, lv - 1));
            if (!dry && ok()) {
                k_tensor(c, A.p, B.p, T3, n, lv, st);
                k_relin_rescale(c, T3, out, n, lv, rs, st);
            }
            pw[k].p = out;
            pw[k].n = n;
            pw[k].L = lv - 1;
            pw[k].scale = P.sc[k];
            pw[k].set = true;
        }
        const uint32_t ls = P.lstar;
        u64* acc = (u64*)take(cts(n, 2, ls));
        u64* tmp = (u64*)take(cts(n, 2, ls));
        void* ss = take(rescale_scratch_bytes(c, n, 2));
        u64* out = (u64*)take(cts(n, 2, ls - 1));
        if (!dry && ok()) {
            fhe_node_const* kc = node_const(i, x.L, x.scale);
            if (!kc) return y;
            bool first = true;
            for (uint32_t k = 1; k <= d; ++k) {
                if (nd.poly[k] == 0.0) continue;
                const u64* Ck = kc->cpow + (size_t)(k - 1) * ls;
                k_mul_const(c, pw[k].p, first ? acc : tmp, n, 2, pw[k].L, ls, Ck, 0, st);
                if (!first) k_add(c, acc, tmp, acc, n, 2, ls, st);
                first = false;
            }
            k_rescale(c, acc, out, n, 2, ls, kc->cpow + (size_t)d * ls, 0, ss, st);
        }
        y.p = out;
        y.n = n;
        y.L = ls - 1;
        y.scale = P.s_y;
        y.set = true;
        return y;
    }

    // ------------------------------------------------ scale schedule of POLY
    struct PolyK {
        int64_t C3 = 0, C2 = 0, C1 = 0, C0 = 0;
        double s_x2 = 0, s_w = 0, s_t1 = 0, s_t2 = 0, s_t3 = 0, s_y = 0;
    };
    PolyK poly_constants(const fhe_graph_node& nd, uint32_t L, double s) const
    {
        PolyK k;
        const double q = (double)c->primes[L - 1];
        if (nd.degree == 1) {
            k.C1 = (int64_t)std::llround(nd.coeffs[1] * q);
            k.s_y = (s * q) / q;
            k.C0 = (int64_t)std::llround(nd.coeffs[0] * k.s_y);
            return k;
        }
        const double qp = (double)c->primes[L - 2];
        const double s2 = (s * s) / q;
        k.s_x2 = (s * s) / q;
        const double s3 = (qp * q) / s2;
        k.C3 = (int64_t)std::llround(nd.coeffs[3] * s3);
        k.s_w = (s * s3) / q;
        k.s_t1 = k.s_x2 * k.s_w;
        const double sg2 = (s * qp) / s2;
        k.C2 = (int64_t)std::llround(nd.coeffs[2] * sg2);
        k.s_t2 = k.s_x2 * sg2;
        k.C1 = (int64_t)std::llround(nd.coeffs[1] * qp);
        k.s_t3 = s * qp;
        k.s_y = (nd.degree == 3 ? k.s_t1 : k.s_t2) / qp;
        k.C0 = (int64_t)std::llround(nd.coeffs[0] * k.s_y);
        return k;
    }

    static bool scale_match(double a, double b) { return std::fabs(a - b) <= std::fabs(a) * std::ldexp(1.0, -40); }

    // ------------------------------------------------ receptors
    Sig linear(uint32_t i, const Sig& x)
    {
        const fhe_graph_node& nd = g->nodes[i];
        Sig y;
        const uint32_t L = x.L;
        if (L < 2) { err(FHE_ELEVEL, "linear node needs two primes"); return y; }
        if (nd.n_out == 0) { err(FHE_EINVAL, "linear node without outputs"); return y; }
        for (uint32_t col : nd.col_idx)
            if (col >= x.n) { err(FHE_EINVAL, "linear column index beyond the stacked input"); return y; }
        const double qd = (double)c->primes[L - 1];
        u64* Y = (u64*)take(cts(nd.n_out, 2, L));
        u64* out = (u64*)take(cts(nd.n_out, 2, L - 1));
        void* sc = take(rescale_scratch_bytes(c, nd.n_out, 2));
        if (!dry && ok()) {
            fhe_node_const* k = node_const(i, L, x.scale);
            if (!k) return y;
            for (int part = 0; part < 2; ++part) {
                const fhe_node_const::TcPart& tp = k->tc[part];
                if (!tp.mask) continue;
                rc = k_linear_mac_tc(c, part == 0 ? 5 : 8, x.p, k->col, k->tc_K, tp.W, tp.rows, tp.tiles, tp.mask, L, Y,
                                     st);
                if (rc != FHE_OK) return y;
            }
            k_linear_mac_tiled(c, x.p, k->tiles, k->n_tiles, k->tile_rows, k->col, k->W, L, Y, st,
                               k->tc[0].mask | k->tc[1].mask, k->max_tile_rows);
            k_rescale(c, Y, out, nd.n_out, 2, L, k->bias, L - 1, sc, st);
        }
        y.p = out;
        y.n = nd.n_out;
        y.L = L - 1;
        y.scale = (x.scale * qd) / qd;
        y.set = true;
        return y;
    }

    Sig square(const Sig& x)
    {
        Sig y;
        const uint32_t L = x.L;
        if (L < 2) { err(FHE_ELEVEL, "square needs two primes"); return y; }
        u64* T3 = (u64*)take(cts(x.n, 3, L));
        void* rs = take(relin_rescale_scratch_bytes(c, x.n, L));
        u64* out = (u64*)take(cts(x.n, 2, L - 1));
        if (!dry && ok()) {
            k_tensor(c, x.p, x.p, T3, x.n, L, st);
            k_relin_rescale(c, T3, out, x.n, L, rs, st);
        }
        y.p = out;
        y.n = x.n;
        y.L = L - 1;
        y.scale = (x.scale * x.scale) / (double)c->primes[L - 1];
        y.set = true;
        return y;
    }

    Sig poly(uint32_t i, const Sig& x)
    {
        Sig y;
        const uint32_t L = x.L, n = x.n;
        const uint32_t deg = g->nodes[i].degree;
        if (deg == 1) return affine(i, x);
        if (deg > 3) return poly_powers(i, x);
        if (L < 3) { err(FHE_ELEVEL, "a degree-2 or -3 activation needs three primes"); return y; }
        const PolyK k = poly_constants(g->nodes[i], L, x.scale);
        if ((deg == 3 && !scale_match(k.s_t1, k.s_t2)) || !scale_match(k.s_t2, k.s_t3)) {
            err(FHE_ESCALE, "polynomial terms disagree in scale");
            return y;
        }
        if (deg == 2) return poly2(i, x, k);
        u64* T3 = (u64*)take(cts(n, 3, L));
        void* rs = take(relin_rescale_scratch_bytes(c, n, L));
        void* ts = take(rescale_tensor_scratch_bytes(c, n, L));
        u64* x2 = (u64*)take(cts(n, 2, L - 1));
        u64* T3b = (u64*)take(cts(n, 3, L - 1));
        u64* out = (u64*)take(cts(n, 2, L - 2));
        if (!dry && ok()) {
            fhe_node_const* kc = node_const(i, L, x.scale);
            if (!kc) return y;
            k_tensor(c, x.p, x.p, T3, n, L, st);
            k_relin_rescale(c, T3, x2, n, L, rs, st);                         // x2 = rescale(relin(x (x) x))
            // x2 (x) w with w = rescale(x * C3), the tensor formed in the rescale's epilogue
            k_rescale_tensor(c, x.p, kc->c3, kc->c3s, x2, T3b, n, L, ts, st);
            // y = rescale(relin(x2 (x) w) + x2 C2 + drop(x) C1) + C0
            const KsExtra ex{x2, kc->c2, kc->c2s, x.p, kc->c1, kc->c1s, (int)L};
            k_relin_rescale(c, T3b, out, n, L - 1, rs, st, &ex, kc->c0, 0);
        }
        y.p = out;
        y.n = n;
        y.L = L - 2;
        y.scale = k.s_y;
        y.set = true;
        return y;
    }

    // degree 1: y = rescale(x * C1) + C0, one fused rescale
    Sig affine(uint32_t i, const Sig& x)
    {
        Sig y;
        const uint32_t L = x.L, n = x.n;
        if (L < 2) { err(FHE_ELEVEL, "an affine activation needs two primes"); return y; }
        const PolyK k = poly_constants(g->nodes[i], L, x.scale);
        void* ss = take(rescale_scratch_bytes(c, n, 2));
        u64* out = (u64*)take(cts(n, 2, L - 1));
        if (!dry && ok()) {
            fhe_node_const* kc = node_const(i, L, x.scale);
            if (!kc) return y;
            k_rescale(c, x.p, out, n, 2, L, kc->c0, 0, ss, st, kc->c1, kc->c1s);
        }
        y.p = out;
        y.n = n;
        y.L = L - 1;
        y.scale = k.s_y;
        y.set = true;
        return y;
    }

    // degree 2: x2 = rescale(relin(x (x) x)); y = rescale(x2 C2 + drop(x) C1) + C0
    Sig poly2(uint32_t i, const Sig& x, const PolyK& k)
    {
        Sig y;
        const uint32_t L = x.L, n = x.n;
        u64* T3 = (u64*)take(cts(n, 3, L));
        void* rs = take(relin_rescale_scratch_bytes(c, n, L));
        void* ss = take(rescale_scratch_bytes(c, n, 2));
        u64* x2 = (u64*)take(cts(n, 2, L - 1));
        u64* t = (u64*)take(cts(n, 2, L - 1));
        u64* out = (u64*)take(cts(n, 2, L - 2));
        if (!dry && ok()) {
            fhe_node_const* kc = node_const(i, L, x.scale);
            if (!kc) return y;
            k_tensor(c, x.p, x.p, T3, n, L, st);
            k_relin_rescale(c, T3, x2, n, L, rs, st);
            k_poly_combine(c, t, x2, x.p, n, L - 1, L, kc->c2, kc->c1, st, false);   // x2 C2 + drop(x) C1
            k_rescale(c, t, out, n, 2, L - 1, kc->c0, 0, ss, st);
        }
        y.p = out;
        y.n = n;
        y.L = L - 2;
        y.scale = k.s_y;
        y.set = true;
        return y;
    }

    // level-match a list of signals by mod-drop (copy of the first L residues)
    Sig drop_to(const Sig& s, uint32_t L)
    {
        if (s.L == L) return s;
        Sig d = s;
        d.L = L;
        d.p = (u64*)take(cts(s.n, 2, L));
        if (!dry && ok()) {
            const size_t w = (size_t)L * c->N * 8, sp = (size_t)s.L * c->N * 8;
            cudaError_t e = cudaMemcpy2DAsync(d.p, w, s.p, sp, w, (size_t)s.n * 2, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) rc = cuda_check(e, "mod-drop copy");
        }
        return d;
    }

    Sig stack(const std::vector<Sig>& in, bool sum)
    {
        Sig y;
        uint32_t Lmin = in[0].L;
        for (const Sig& s : in) Lmin = std::min(Lmin, s.L);
        std::vector<Sig> m;
        for (const Sig& s : in) m.push_back(drop_to(s, Lmin));
        for (const Sig& s : m)
            if (!scale_match(m[0].scale, s.scale)) { err(FHE_ESCALE, "stacked inputs disagree in scale"); return y; }
        if (sum) {
            for (const Sig& s : m)
                if (s.n != m[0].n) { err(FHE_EINVAL, "add node inputs differ in length"); return y; }
            u64* out = (u64*)take(cts(m[0].n, 2, Lmin));
            if (!dry && ok()) {
                k_add(c, m[0].p, m[1].p, out, m[0].n, 2, Lmin, st);
                for (size_t k = 2; k < m.size(); ++k) k_add(c, out, m[k].p, out, m[0].n, 2, Lmin, st);
            }
            y.p = out;
            y.n = m[0].n;
        } else {
            uint32_t n = 0;
            for (const Sig& s : m) n += s.n;
            u64* out = (u64*)take(cts(n, 2, Lmin));
            if (!dry && ok()) {
                size_t off = 0;
                for (const Sig& s : m) {
                    cudaError_t e = cudaMemcpyAsync(out + off, s.p, cts(s.n, 2, Lmin), cudaMemcpyDeviceToDevice, st);
                    if (e != cudaSuccess) rc = cuda_check(e, "stack copy");
                    off += cts(s.n, 2, Lmin) / 8;
                }
            }
            y.p = out;
            y.n = n;
        }
        y.L = Lmin;
        y.scale = m[0].scale;
        y.set = true;
        return y;
    }

    // ------------------------------------------------ Alg. firing
    bool inbound(uint32_t n, const Sig* bootstrap, Sig* s)
    {
        if (bootstrap) {
            *s = *bootstrap;
            return true;
        }
        std::vector<Sig> in;
        for (uint32_t e : in_e[n]) {
            if (!edge[e].set) return false;
            in.push_back(edge[e]);
        }
        if (in.empty()) return false;
        if (in.size() == 1) {
            *s = in[0];
            return true;
        }
        *s = stack(in, g->nodes[n].kind == FHE_NODE_ADD);
        return s->set;
    }

    Sig apply(uint32_t n, const Sig& s)
    {
        switch (g->nodes[n].kind) {
        case FHE_NODE_INPUT:
        case FHE_NODE_OUTPUT:
        case FHE_NODE_ADD: return s;
        case FHE_NODE_LINEAR: return linear(n, s);
        case FHE_NODE_SQUARE: return square(s);
        case FHE_NODE_POLY:
        case FHE_NODE_RELU: return poly(n, s);
        case FHE_NODE_CONV_PACKED: return conv_packed(n, s);
        case FHE_NODE_ROTATE:
            err(FHE_EUNSUPPORTED, "a rotation node hands its ciphertexts to the client: evaluate each parameter group "
                                  "on its own context");
            return Sig();
        default: err(FHE_EINVAL, "unknown node kind"); return Sig();
        }
    }

    void carrier(uint32_t n, const Sig* bootstrap, int depth)
    {
        if (!ok() || fired[n]) return;
        if (depth > 10000) { err(FHE_EINVAL, "graph too deep"); return; }
        Sig s;
        if (!inbound(n, bootstrap, &s)) return;
        s = apply(n, s);
        if (!ok() || !s.set) return;
        fired[n] = 1;
        if (g->nodes[n].kind == FHE_NODE_OUTPUT) outputs[n] = s;
        for (uint32_t e : out_e[n]) edge[e] = s;
        std::vector<uint32_t> seen;
        for (uint32_t e : out_e[n]) {
            const uint32_t b = g->edst[e];
            if (std::find(seen.begin(), seen.end(), b) != seen.end()) continue;
            seen.push_back(b);
            carrier(b, nullptr, depth + 1);
        }
    }

    void run(const uint64_t* const* d_in, uint32_t n_inputs)
    {
        const uint32_t nn = (uint32_t)g->nodes.size();
        edge.assign(g->esrc.size(), Sig());
        fired.assign(nn, 0);
        outputs.assign(nn, Sig());
        in_e.assign(nn, {});
        out_e.assign(nn, {});
        for (uint32_t e = 0; e < g->esrc.size(); ++e) {
            out_e[g->esrc[e]].push_back(e);
            in_e[g->edst[e]].push_back(e);
        }
        uint32_t k = 0;
        for (uint32_t n = 0; n < nn && ok(); ++n) {
            if (g->nodes[n].kind != FHE_NODE_INPUT) continue;
            if (k >= n_inputs) { err(FHE_EINVAL, "fewer input buffers than input nodes"); return; }
            Sig s;
            s.p = d_in ? (u64*)d_in[k] : nullptr;
            s.n = g->nodes[n].n_out;
            s.L = c->L_top;
            s.scale = c->delta;
            s.set = true;
            ++k;
            carrier(n, &s, 0);
        }
        if (ok() && k != n_inputs) err(FHE_EINVAL, "more input buffers than input nodes");
    }
};

}  // namespace

extern "C" {

int fhe_graph_create(const fhe_graph_desc* d, fhe_graph** out)
{
    if (!d || !out || (!d->nodes && d->n_nodes)) return fail(FHE_EINVAL, "null graph description");
    *out = nullptr;
    fhe_graph* g = new fhe_graph();
    for (uint32_t i = 0; i < d->n_nodes; ++i) {
        const fhe_node_desc& s = d->nodes[i];
        fhe_graph_node n;
        n.kind = s.kind;
        n.n_out = s.n_out;
        if (s.kind > FHE_NODE_CONV_PACKED) {
            delete g;
            return fail(FHE_EINVAL, "unknown node kind");
        }
        if (s.kind == FHE_NODE_LINEAR) {
            if (!s.row_ptr || (s.n_out && (!s.col_idx || !s.weight))) {
                delete g;
                return fail(FHE_EINVAL, "linear node without CSR arrays");
            }
            n.row_ptr.assign(s.row_ptr, s.row_ptr + s.n_out + 1);
            const uint32_t nnz = n.row_ptr.back();
            if (n.row_ptr[0] != 0) {
                delete g;
                return fail(FHE_EINVAL, "row_ptr[0] must be 0");
            }
            for (uint32_t o = 0; o < s.n_out; ++o) {
                if (n.row_ptr[o + 1] < n.row_ptr[o]) {
                    delete g;
                    return fail(FHE_EINVAL, "row_ptr must be non-decreasing");
                }
                if (n.row_ptr[o + 1] - n.row_ptr[o] >= (1u << 20)) {     // exact 64-bit limb sums
                    delete g;
                    return fail(FHE_EUNSUPPORTED, "a linear row has 2^20 or more terms");
                }
            }
            n.col_idx.assign(s.col_idx, s.col_idx + nnz);
            n.weight.assign(s.weight, s.weight + nnz);
            if (s.bias) n.bias.assign(s.bias, s.bias + s.n_out);
            else n.bias.assign(s.n_out, 0.0);
            for (double w : n.weight)
                if (!std::isfinite(w)) {
                    delete g;
                    return fail(FHE_EINVAL, "non-finite weight");
                }
        }
        for (int k = 0; k < 4; ++k) n.coeffs[k] = s.coeffs[k];
        if (s.kind == FHE_NODE_CONV_PACKED) {
            for (int k = 0; k < 6; ++k) n.conv[k] = s.conv[k];
            const uint32_t H = n.conv[0], W = n.conv[1], k = n.conv[2], st_ = n.conv[3], imgs = n.conv[4],
                           S = n.conv[5];
            if (!s.n_out || !s.weight || !k || !st_ || !imgs || k > H || k > W || S < H * W) {
                delete g;
                return fail(FHE_EINVAL, "packed convolution: bad geometry or missing weights");
            }
            n.weight.assign(s.weight, s.weight + (size_t)s.n_out * k * k);
            if (s.bias) n.bias.assign(s.bias, s.bias + s.n_out);
            else n.bias.assign(s.n_out, 0.0);
        }
        if (s.kind == FHE_NODE_POLY) {
            n.degree = s.degree == 0 ? 3 : s.degree;
            if (n.degree > kMaxPolyDegree) {
                delete g;
                return fail(FHE_EUNSUPPORTED, "polynomial degree above 31");
            }
            if (n.degree > 3) {
                if (!s.coeffs_hi) {
                    delete g;
                    return fail(FHE_EINVAL, "a polynomial of degree above 3 needs coeffs_hi");
                }
                n.poly.assign(s.coeffs_hi, s.coeffs_hi + n.degree + 1);
                bool any = false;
                for (uint32_t k = 1; k <= n.degree; ++k) any |= n.poly[k] != 0.0;
                if (!any) {
                    delete g;
                    return fail(FHE_EINVAL, "polynomial without non-constant terms");
                }
            }
            for (uint32_t k = n.degree + 1; k < 4; ++k) n.coeffs[k] = 0.0;
        } else if (s.kind == FHE_NODE_RELU) {
            // Eq. relu_approximate with range q, as a degree-2 polynomial
            const double q = s.coeffs[0];
            if (!(q > 0.0) || !std::isfinite(q)) {
                delete g;
                return fail(FHE_EINVAL, "ReLU approximation range q must be positive");
            }
            n.degree = 2;
            n.coeffs[0] = q / (3 * M_PI);
            n.coeffs[1] = 0.5;
            n.coeffs[2] = 4 / (3 * M_PI * q);
            n.coeffs[3] = 0.0;
        }
        g->nodes.push_back(n);
    }
    for (uint32_t e = 0; e < d->n_edges; ++e) {
        if (d->edge_src[e] >= d->n_nodes || d->edge_dst[e] >= d->n_nodes) {
            delete g;
            return fail(FHE_EINVAL, "edge endpoint out of range");
        }
        g->esrc.push_back(d->edge_src[e]);
        g->edst.push_back(d->edge_dst[e]);
    }
    g->cache.resize(g->nodes.size());
    *out = g;
    return FHE_OK;
}

int fhe_graph_destroy(fhe_graph* g)
{
    if (!g) return FHE_OK;
    bool any = false;
    for (auto& nc : g->cache) any |= (nc.buf != nullptr);
    if (any) cudaDeviceSynchronize();
    for (auto& nc : g->cache) cudaFree(nc.buf);
    delete g;
    return FHE_OK;
}

static int dry_run(fhe_ctx* c, fhe_graph* g, uint32_t n_inputs, Exec* X)
{
    X->c = c;
    X->g = g;
    X->st = nullptr;
    X->dry = true;
    X->run(nullptr, n_inputs);
    return X->rc;
}

static int count_inputs(const fhe_graph* g)
{
    int k = 0;
    for (const auto& n : g->nodes) k += (n.kind == FHE_NODE_INPUT);
    return k;
}

int fhe_graph_outputs(fhe_ctx* c, const fhe_graph* gc, uint32_t* n_out_cts, uint32_t* out_level)
{
    if (!c || !gc) return fail(FHE_EINVAL, "null argument");
    fhe_graph* g = const_cast<fhe_graph*>(gc);
    Exec X;
    int rc = dry_run(c, g, (uint32_t)count_inputs(g), &X);
    if (rc) return rc;
    uint32_t n = 0, L = 0;
    bool first = true;
    for (size_t i = 0; i < g->nodes.size(); ++i) {
        if (g->nodes[i].kind != FHE_NODE_OUTPUT) continue;
        if (!X.outputs[i].set) return fail(FHE_EINVAL, "an output node never fires");
        n += X.outputs[i].n;
        L = first ? X.outputs[i].L : std::min(L, X.outputs[i].L);
        first = false;
    }
    if (n_out_cts) *n_out_cts = n;
    if (out_level) *out_level = L;
    return FHE_OK;
}

int fhe_eval_graph(fhe_ctx* c, const fhe_graph* gc, const uint64_t* const* d_in, uint32_t n_inputs, uint64_t* d_out,
                   fhe_ct_meta* out_meta, uint32_t out_cap, void* stream)
{
    if (!c || !gc || !d_in || !d_out) return fail(FHE_EINVAL, "null argument");
    if (!c->has_keys) return fail(FHE_ENOKEY, "fhe_keygen has not run");
    fhe_graph* g = const_cast<fhe_graph*>(gc);
    const fhe_ctx* root = c->parent ? c->parent : c;     // forks share the primes
    if (g->cache_ctx != root) {
        bool any = false;
        for (auto& nc : g->cache) any |= (nc.buf != nullptr);
        if (any) cudaDeviceSynchronize();
        for (auto& nc : g->cache) {
            cudaFree(nc.buf);
            nc = fhe_node_const();
        }
        g->cache_ctx = root;
    }
    for (uint32_t i = 0; i < n_inputs; ++i)
        if (!d_in[i]) return fail(FHE_EINVAL, "null input buffer");
    Exec D;
    int rc = dry_run(c, g, n_inputs, &D);
    if (rc) return rc;
    uint32_t n_out = 0, Lout = 0;
    bool first = true;
    for (size_t i = 0; i < g->nodes.size(); ++i) {
        if (g->nodes[i].kind != FHE_NODE_OUTPUT) continue;
        if (!D.outputs[i].set) return fail(FHE_EINVAL, "an output node never fires");
        n_out += D.outputs[i].n;
        Lout = first ? D.outputs[i].L : std::min(Lout, D.outputs[i].L);
        first = false;
    }
    if (n_out > out_cap) return fail(FHE_EINVAL, "out_cap smaller than the number of output ciphertexts");

    Exec X;
    X.c = c;
    X.g = g;
    X.st = (cudaStream_t)stream;
    X.dry = false;
    rc = ws_reserve(c, D.need, &X.ar);
    if (rc) return rc;
    X.run(d_in, n_inputs);
    if (X.rc) return X.rc;
    size_t off = 0;
    const size_t N = c->N;
    for (size_t i = 0; i < g->nodes.size(); ++i) {
        if (g->nodes[i].kind != FHE_NODE_OUTPUT) continue;
        const Sig& s = X.outputs[i];
        const size_t w = (size_t)Lout * N * 8, sp = (size_t)s.L * N * 8;
        cudaError_t e = cudaMemcpy2DAsync((char*)d_out + off, w, s.p, sp, w, (size_t)s.n * 2, cudaMemcpyDeviceToDevice,
                                          X.st);
        if (e != cudaSuccess) return cuda_check(e, "output copy");
        off += (size_t)s.n * 2 * w;
        if (out_meta) {
            size_t base = 0;
            for (size_t j = 0; j < i; ++j)
                if (g->nodes[j].kind == FHE_NODE_OUTPUT) base += X.outputs[j].n;
            for (uint32_t k = 0; k < s.n; ++k) {
                out_meta[base + k].level = Lout;
                out_meta[base + k].scale = s.scale;
            }
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(e, "graph launch");
    return status_take(c);
}

}  // extern "C"
