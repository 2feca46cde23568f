// H_eff*psi without any device allocation, for callers that must not allocate GPU
// memory themselves: a process whose device memory is owned and budgeted by a host
// framework's allocator (an extra cudaMalloc would escape its accounting or fail once
// its pool holds the memory), or a plugin embedded in another application that only
// receives device buffers.  The call is synchronous with respect to its stream's
// earlier work (it waits for the staged tables to land), so it is meant for set-up,
// checking and fallback use rather than for a tight loop.
//
// The caller passes the inputs and the output; everything else this path needs (the
// staged term tables and one intermediate block per CTA) lives in the fixed file-scope
// array below, which exists once per GPU that loads the library and stays resident
// until the process exits.  All calls share it: calls from several host threads are
// serialised per device from the staging of the tables to the kernel launch, but calls
// whose work overlaps on the GPU (two streams without ordering) race with each other.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/dmrg_heff.h"
#include "handle.h"

namespace dmrg {
namespace {

constexpr size_t NOALLOC_BYTES = size_t(DMRG_NOALLOC_SCRATCH_BYTES);
constexpr int NOALLOC_MAX_SECTORS = 512;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

struct NaBlock { int64_t off; int32_t rows, cols, iR, pad; };   // psi block whose left sector is i

struct NaArgs {
    const int32_t* left;
    const int32_t* right;
    const NaBlock* blk;
    const double* coef;
    const int32_t* delta;
    const int32_t* parity;
    const int64_t* a_off;
    const int64_t* b_off;
    double* xbuf;          // per-CTA intermediate blocks
    int64_t xbuf_len;      // doubles per CTA
    int32_t nl, nr, T, pad;
    const double* op;
    const double* x;
    double* y;
};

__device__ int na_find(const int32_t* tab, int n, int32_t q, int32_t s) {
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int32_t mq = tab[3 * mid], ms = tab[3 * mid + 1];
        if (mq == q && ms == s) return mid;
        if (mq < q || (mq == q && ms < s)) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// One CTA owns whole output blocks: y_o = sum_t c_t s_t A_t (x_q) B_t^T, with the
// intermediate X = A_t x_q (rows x c) in the CTA's part of the static array; terms are
// taken in order, so the result does not depend on the launch configuration.
__global__ void __launch_bounds__(256) k_heff_noalloc(NaArgs a) {
    double* X = a.xbuf + int64_t(blockIdx.x) * a.xbuf_len;
    for (int o = blockIdx.x; o < a.nl; o += gridDim.x) {
        const NaBlock O = a.blk[o];
        if (O.iR < 0) continue;
        double* yo = a.y + O.off;
        for (int e = threadIdx.x; e < O.rows * O.cols; e += blockDim.x) yo[e] = 0.0;
        __syncthreads();
        for (int t = 0; t < a.T; ++t) {
            const int32_t dn = a.delta[2 * t], ds = a.delta[2 * t + 1];
            const int qL = na_find(a.left, a.nl, a.left[3 * o] - dn, a.left[3 * o + 1] - ds);
            if (qL < 0) continue;
            const NaBlock Q = a.blk[qL];
            if (Q.iR < 0) continue;
            const int64_t ao = a.a_off[int64_t(t) * a.nl + qL], bo = a.b_off[int64_t(t) * a.nr + Q.iR];
            if (ao < 0 || bo < 0) continue;
            const int b = Q.rows, c = Q.cols;
            const double* A = a.op + ao;      // O.rows x b
            const double* B = a.op + bo;      // O.cols x c
            const double* xq = a.x + Q.off;   // b x c
            const double s = (a.parity[t] && (a.left[3 * qL] & 1)) ? -a.coef[t] : a.coef[t];
            for (int e = threadIdx.x; e < O.rows * c; e += blockDim.x) {
                const int i = e / c, j = e % c;
                double acc = 0.0;
                for (int k = 0; k < b; ++k) acc += A[int64_t(i) * b + k] * xq[int64_t(k) * c + j];
                X[e] = acc;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < O.rows * O.cols; e += blockDim.x) {
                const int i = e / O.cols, j = e % O.cols;
                double acc = 0.0;
                for (int k = 0; k < c; ++k) acc += X[int64_t(i) * c + k] * B[int64_t(j) * c + k];
                yo[e] += s * acc;
            }
            __syncthreads();
        }
    }
}

std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[NOALLOC_MAX_DEVICES] = {};
// Per device: held from the first table copy into the array to the kernel launch, so
// that two host threads on one stream cannot interleave their copies and kernels.
std::mutex g_call_mutex[NOALLOC_MAX_DEVICES];

// Device address of the static array on the current device, looked up once per device.
int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(DMRG_ERR_UNSUPPORTED, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return DMRG_OK;
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace
}  // namespace dmrg

extern "C" int dmrg_heff_apply_noalloc(const int32_t* left, int32_t nl, const int32_t* right, int32_t nr,
                                       int32_t target_n, int32_t target_2sz, const double* coef,
                                       const int32_t* delta, const int32_t* parity, const int64_t* a_off,
                                       const int64_t* b_off, int64_t n_terms, const double* op_data,
                                       int64_t op_len, const double* x, double* y, void* stream) {
    using namespace dmrg;
    if (nl < 0 || nr < 0 || n_terms < 0 || op_len < 0) return fail(DMRG_ERR_INVALID_ARG, "negative size");
    if (nl > NOALLOC_MAX_SECTORS || nr > NOALLOC_MAX_SECTORS)
        return fail(DMRG_ERR_INVALID_ARG, "more than 512 sectors per block: beyond the no-allocation path");
    if (n_terms > (int64_t(1) << 24)) return fail(DMRG_ERR_INVALID_ARG, "too many terms");
    if ((nl && !left) || (nr && !right) ||
        (n_terms && (!coef || !delta || !parity || (nl && !a_off) || (nr && !b_off))))
        return fail(DMRG_ERR_INVALID_ARG, "null host array");
    auto sorted = [](const int32_t* t, int32_t n) {
        for (int32_t i = 0; i < n; ++i) {
            if (t[3 * i + 2] < 1) return false;
            if (i && !(t[3 * i - 3] < t[3 * i] || (t[3 * i - 3] == t[3 * i] && t[3 * i - 2] < t[3 * i + 1]))) return false;
        }
        return true;
    };
    if (!sorted(left, nl) || !sorted(right, nr))
        return fail(DMRG_ERR_INVALID_ARG, "sector tables must be strictly ascending with dims >= 1");
    auto find = [](const int32_t* t, int32_t n, int32_t q, int32_t s) {
        for (int32_t i = 0; i < n; ++i)
            if (t[3 * i] == q && t[3 * i + 1] == s) return i;
        return -1;
    };
    // wave-function blocks (host stack only)
    NaBlock blk[NOALLOC_MAX_SECTORS];
    int64_t dim = 0, max_dl = 0, max_dr = 0;
    for (int32_t i = 0; i < nl; ++i) {
        const int j = find(right, nr, target_n - left[3 * i], target_2sz - left[3 * i + 1]);
        blk[i] = {dim, left[3 * i + 2], j >= 0 ? right[3 * j + 2] : 0, j, 0};
        if (j >= 0) dim += int64_t(left[3 * i + 2]) * right[3 * j + 2];
        if (left[3 * i + 2] > max_dl) max_dl = left[3 * i + 2];
    }
    for (int32_t j = 0; j < nr; ++j)
        if (right[3 * j + 2] > max_dr) max_dr = right[3 * j + 2];
    // operator offsets: present blocks must have their output sector and fit in op_data
    for (int64_t t = 0; t < n_terms; ++t) {
        if (parity[t] != 0 && parity[t] != 1) return fail(DMRG_ERR_INVALID_ARG, "parity flag must be 0 or 1");
        for (int32_t q = 0; q < nl; ++q) {
            const int64_t o = a_off[t * nl + q];
            if (o == -1) continue;
            const int p = find(left, nl, left[3 * q] + delta[2 * t], left[3 * q + 1] + delta[2 * t + 1]);
            if (p < 0) return fail(DMRG_ERR_SECTOR_MISMATCH, "A block present for an absent output sector");
            if (o < 0 || int64_t(left[3 * p + 2]) * left[3 * q + 2] > op_len - o)
                return fail(DMRG_ERR_INVALID_ARG, "A block offset out of range");
        }
        for (int32_t q = 0; q < nr; ++q) {
            const int64_t o = b_off[t * nr + q];
            if (o == -1) continue;
            const int p = find(right, nr, right[3 * q] - delta[2 * t], right[3 * q + 1] - delta[2 * t + 1]);
            if (p < 0) return fail(DMRG_ERR_SECTOR_MISMATCH, "B block present for an absent output sector");
            if (o < 0 || int64_t(right[3 * p + 2]) * right[3 * q + 2] > op_len - o)
                return fail(DMRG_ERR_INVALID_ARG, "B block offset out of range");
        }
    }
    if (dim == 0) return DMRG_OK;
    if (!op_data || !x || !y) return fail(DMRG_ERR_INVALID_ARG, "null device pointer");
    {
        const char* xb = reinterpret_cast<const char*>(x);
        const char* yb = reinterpret_cast<const char*>(y);
        const size_t bytes = sizeof(double) * size_t(dim);
        if (xb < yb + bytes && yb < xb + bytes) return fail(DMRG_ERR_INVALID_ARG, "x and y overlap");
    }
    // layout of the static array: tables, then one intermediate block per CTA
    const size_t T = size_t(n_terms);
    size_t off = 0;
    const size_t o_left = off; off = align256(off + 12 * size_t(nl));
    const size_t o_right = off; off = align256(off + 12 * size_t(nr));
    const size_t o_blk = off; off = align256(off + sizeof(NaBlock) * size_t(nl));
    const size_t o_coef = off; off = align256(off + 8 * T);
    const size_t o_delta = off; off = align256(off + 8 * T);
    const size_t o_par = off; off = align256(off + 4 * T);
    const size_t o_aoff = off; off = align256(off + 8 * T * size_t(nl));
    const size_t o_boff = off; off = align256(off + 8 * T * size_t(nr));
    const size_t xlen = size_t(max_dl * max_dr);
    const size_t per_cta = align256(8 * xlen);
    if (off + per_cta > NOALLOC_BYTES)
        return fail(DMRG_ERR_INVALID_ARG, "problem needs more than the 32 MiB static scratch of the no-allocation path");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    int64_t grid = int64_t(nl);
    if (grid > 2 * int64_t(sms)) grid = 2 * int64_t(sms);
    const int64_t fit = int64_t((NOALLOC_BYTES - off) / per_cta);
    if (grid > fit) grid = fit;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the call synchronises its stream (below), which a capturing stream does not allow:
    // refuse before touching the stream, so that the caller's capture stays valid
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "stream query");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(DMRG_ERR_UNSUPPORTED, "the stream is capturing; this call synchronises its stream");
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != DMRG_OK) return rc;
    std::lock_guard<std::mutex> call_lock(g_call_mutex[dev]);
    struct Copy { size_t off; const void* src; size_t bytes; } copies[] = {
        {o_left, left, 12 * size_t(nl)},       {o_right, right, 12 * size_t(nr)},
        {o_blk, blk, sizeof(NaBlock) * nl},    {o_coef, coef, 8 * T},
        {o_delta, delta, 8 * T},               {o_par, parity, 4 * T},
        {o_aoff, a_off, 8 * T * size_t(nl)},   {o_boff, b_off, 8 * T * size_t(nr)}};
    for (const Copy& c : copies) {
        if (c.bytes == 0) continue;
        e = cudaMemcpyAsync(base + c.off, c.src, c.bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "stage tables into the static scratch");
    }
    // the staged block table lives on this host stack frame; make sure it has been read
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "stage tables");
    NaArgs args;
    args.left = reinterpret_cast<const int32_t*>(base + o_left);
    args.right = reinterpret_cast<const int32_t*>(base + o_right);
    args.blk = reinterpret_cast<const NaBlock*>(base + o_blk);
    args.coef = reinterpret_cast<const double*>(base + o_coef);
    args.delta = reinterpret_cast<const int32_t*>(base + o_delta);
    args.parity = reinterpret_cast<const int32_t*>(base + o_par);
    args.a_off = reinterpret_cast<const int64_t*>(base + o_aoff);
    args.b_off = reinterpret_cast<const int64_t*>(base + o_boff);
    args.xbuf = reinterpret_cast<double*>(base + off);
    args.xbuf_len = int64_t(per_cta / 8);
    args.nl = nl; args.nr = nr; args.T = int32_t(n_terms); args.pad = 0;
    args.op = op_data; args.x = x; args.y = y;
    k_heff_noalloc<<<unsigned(grid), 256, 0, st>>>(args);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation kernel");
    return DMRG_OK;
}
