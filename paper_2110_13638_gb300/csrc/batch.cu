// batch.cu -- fhe_eval_batch: one served batch of encrypted-inference
// requests, packed into the slots of one set of input ciphertexts and run
// through the graph on one stream.
#include <string>
#include <vector>

#include "../../include/fhe.h"
#include "ctx.h"

using namespace fhe;

namespace {

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

int bb_reserve(fhe_ctx* c, size_t bytes)
{
    if (c->bb_bytes >= bytes) return FHE_OK;
    if (c->bb) {
        cudaDeviceSynchronize();       // earlier batches may still read the area
        cudaFree(c->bb);
        c->bb = nullptr;
        c->bb_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&c->bb, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_check(e, "batch area cudaMalloc");
    }
    c->bb_bytes = bytes;
    return FHE_OK;
}

}  // namespace

extern "C" int fhe_eval_batch(fhe_ctx* c, const fhe_graph* g, const fhe_request* reqs, uint32_t n_reqs,
                              uint64_t first_ct_id, void* stream)
{
    if (!c || !g) return fail(FHE_EINVAL, "null argument");
    if (!c->has_keys) return fail(FHE_ENOKEY, "fhe_keygen has not run");
    if (n_reqs > 0 && !reqs) return fail(FHE_EINVAL, "null request array");
    uint32_t n_in = 0, inputs = 0;
    for (const auto& nd : g->nodes)
        if (nd.kind == FHE_NODE_INPUT) {
            ++inputs;
            n_in = nd.n_out;
        }
    if (inputs != 1) return fail(FHE_EINVAL, "fhe_eval_batch needs a graph with exactly one INPUT node");
    if (n_in == 0) return fail(FHE_EINVAL, "the INPUT node receives no ciphertexts");
    const size_t N = c->N, M = N / 2;
    size_t total = 0;
    for (uint32_t k = 0; k < n_reqs; ++k) {
        const fhe_request& r = reqs[k];
        if (r.n_samples == 0 || !r.x || !r.y) return fail(FHE_EINVAL, "request without samples or buffers");
        if (r.x_stride < r.n_samples || r.y_stride < r.n_samples) return fail(FHE_EINVAL, "request stride below n_samples");
        total += r.n_samples;
    }
    if (total > M)
        return fail(FHE_EINVAL, "requests hold " + std::to_string(total) + " samples; one batch has " +
                                    std::to_string(M) + " slots");
    if (n_reqs == 0) return FHE_OK;
    uint32_t n_out = 0, L_out = 0;
    int rc = fhe_graph_outputs(c, g, &n_out, &L_out);
    if (rc) return rc;
    const uint32_t Lt = c->L_top;
    const size_t b_slots = al256((size_t)n_in * M * 8), b_ct = al256((size_t)n_in * 2 * Lt * N * 8);
    const size_t b_out = al256((size_t)n_out * 2 * L_out * N * 8), b_m = al256((size_t)n_out * N * 8);
    const size_t b_z = al256((size_t)n_out * M * 8);
    rc = bb_reserve(c, b_slots + b_ct + b_out + b_m + b_z);
    if (rc) return rc;
    char* p = (char*)c->bb;
    double* slots = (double*)p;
    uint64_t* ct = (uint64_t*)(p + b_slots);
    uint64_t* out = (uint64_t*)(p + b_slots + b_ct);
    int64_t* m = (int64_t*)(p + b_slots + b_ct + b_out);
    double* z = (double*)(p + b_slots + b_ct + b_out + b_m);
    cudaStream_t st = (cudaStream_t)stream;

    // gather: request k -> columns [off_k, off_k + n_k) of every input row
    cudaError_t e = cudaSuccess;
    if (total < M)
        e = cudaMemset2DAsync(slots + total, M * 8, 0, (M - total) * 8, n_in, st);
    size_t off = 0;
    for (uint32_t k = 0; k < n_reqs && e == cudaSuccess; ++k) {
        const fhe_request& r = reqs[k];
        e = cudaMemcpy2DAsync(slots + off, M * 8, r.x, (size_t)r.x_stride * 8, (size_t)r.n_samples * 8, n_in,
                              cudaMemcpyDefault, st);
        off += r.n_samples;
    }
    if (e != cudaSuccess) return cuda_check(e, "batch gather");

    rc = fhe_encode_encrypt(c, slots, n_in, c->delta, first_ct_id, ct, stream);
    if (rc) return rc;
    std::vector<fhe_ct_meta> meta(n_out);
    const uint64_t* ins[1] = {ct};
    rc = fhe_eval_graph(c, g, ins, 1, out, meta.data(), n_out, stream);
    if (rc) return rc;
    rc = fhe_decrypt(c, out, n_out, L_out, m, stream);
    if (rc) return rc;
    // decode each run of outputs that share a nominal scale
    for (uint32_t a = 0; a < n_out;) {
        uint32_t b = a + 1;
        while (b < n_out && meta[b].scale == meta[a].scale) ++b;
        rc = fhe_decode(c, m + (size_t)a * N, b - a, meta[a].scale, z + (size_t)a * M, stream);
        if (rc) return rc;
        a = b;
    }
    // scatter: columns of request k -> its y rows
    off = 0;
    for (uint32_t k = 0; k < n_reqs && e == cudaSuccess; ++k) {
        const fhe_request& r = reqs[k];
        e = cudaMemcpy2DAsync(r.y, (size_t)r.y_stride * 8, z + off, M * 8, (size_t)r.n_samples * 8, n_out,
                              cudaMemcpyDefault, st);
        off += r.n_samples;
    }
    if (e != cudaSuccess) return cuda_check(e, "batch scatter");
    return status_take(c);
}
