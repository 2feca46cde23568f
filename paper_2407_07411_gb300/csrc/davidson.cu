// Block Davidson on the device (the local eigenproblem of each DMRG update, solved by
// Lanczos or Davidson after Eq. 2 of the paper).  All vector arithmetic is FP64 in the
// kernels below; H_eff*psi is the handle's apply (FP64 or split precision).  The host
// loop only sequences launches and reads back a few scalars per step (Ritz values,
// residual norms, CGS2 norms), so the steps mirror the documented variant exactly:
//
//   Rayleigh-Ritz on S = sym(V W^T) by cyclic Jacobi (one CTA, parallel ordering),
//   Ritz vectors / residuals for the lowest kb = min(m, max(k_eig, b)) pairs,
//   corrections r / (diag - theta) (|den| < 1e-8 -> +-1e-8) for the first b
//   unconverged pairs, thick restart to k_eig + b Ritz vectors when the basis is full,
//   CGS2 (two classical Gram-Schmidt passes, drop below 1e-10 of the input norm).
#include <chrono>
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/dmrg_heff.h"
#include "handle.h"
#include "jacobi_rot.cuh"

namespace dmrg {

// Dot products are cut into chunks of at least DOT_MIN_CHUNK elements, about two per SM
// on large vectors (FP64 arithmetic is scarce on this GPU, so every SM takes a share);
// a chunk gives each thread at least 16 elements, so that a CTA's reduction (FP64 work
// too) stays small against its products.  Partials are summed in a fixed order.
constexpr int DOT_MIN_CHUNK = 4096;
constexpr int DOT_NT = 256;
constexpr int MAXQ = 8;          // Q vectors per multi-dot launch
constexpr int MAX_BASIS = 64;    // m_max limit of the Jacobi kernel

struct DavidsonState {
    double *V = nullptr, *W = nullptr, *X = nullptr, *R = nullptr, *C = nullptr, *T = nullptr;
    double *diag = nullptr, *S = nullptr, *U = nullptr, *theta = nullptr, *small = nullptr, *partial = nullptr;
    unsigned* done = nullptr;          // completion count of the dot-product kernel (zero between launches)
    int64_t n_chunks = 0, chunk = 0;   // dot-product partials: count and length
    int mmax = 0, kbmax = 0, block = 0, k_eig = 0;   // sizes the buffers were allocated for
    bool diag_ready = false;
    ~DavidsonState() {
        double* p[] = {V, W, X, R, C, T, diag, S, U, theta, small, partial};
        for (double* q : p)
            if (q) cudaFree(q);
        if (done) cudaFree(done);
    }
};

namespace {

// Sum over the warp in a fixed shuffle tree (the result in lane 0).  FP64 additions are
// long-latency operations on this GPU: reductions use shuffle trees over many lanes
// instead of long chains in one thread.
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// Sum over the CTA of DOT_NT threads (fixed order: warp trees, then a shuffle tree over
// the warps' sums in warp 0); the result in thread 0.  red holds DOT_NT / 32 doubles.
__device__ __forceinline__ double cta_sum(double x, double* red) {
    x = warp_sum(x);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < DOT_NT / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = DOT_NT / 64; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;
}

// out[i*nq + j] = P_i . Q_j: partial[(c*np + i)*nq + j] = sum over chunk c (fixed-order
// tree), then the CTA that finishes last (a counter, reset by that CTA for the next
// launch) adds the chunks' partials in a fixed order (a warp per output), so the result
// does not depend on which CTA runs when.  With gridDim.z = 2 the same is done for out2 = P2 . Q2 (CTAs of
// z = 1), and with S given the last CTA also writes the symmetric Rayleigh-Ritz entries
// S[i][m0 + j] = S[m0 + j][i] = (out[i*nq + j] + out2[i*nq + j]) / 2.
// nq is a template parameter: an FP64 instruction whose predicate is off still holds the
// FP64 pipe on this GPU, so the loops over the Q vectors have exactly nq iterations.
template <int nq>
__global__ void __launch_bounds__(DOT_NT) k_multidot(const double* __restrict__ P, int64_t ldp, int np,
                                                     const double* __restrict__ Q, int64_t ldq,
                                                     int64_t dim, int64_t chunk, double* __restrict__ partial,
                                                     double* __restrict__ out, unsigned* __restrict__ done,
                                                     const double* __restrict__ P2, const double* __restrict__ Q2,
                                                     double* __restrict__ out2, double* __restrict__ S, int lds,
                                                     int m0) {
    __shared__ double red[DOT_NT / 32];
    __shared__ bool last;
    const int c = blockIdx.x, i = blockIdx.y, z = blockIdx.z;
    const int npq = np * nq;
    const int64_t n0 = int64_t(c) * chunk;
    const int64_t n1 = min(dim, n0 + chunk);
    double acc[nq];
#pragma unroll
    for (int j = 0; j < nq; ++j) acc[j] = 0.0;
    const double* p = (z ? P2 : P) + i * ldp;
    const double* Qz = z ? Q2 : Q;
    for (int64_t n = n0 + threadIdx.x; n < n1; n += DOT_NT) {
        const double pv = p[n];
#pragma unroll
        for (int j = 0; j < nq; ++j) acc[j] += pv * Qz[j * ldq + n];
    }
    double* part = partial + int64_t(z) * gridDim.x * npq;
#pragma unroll
    for (int j = 0; j < nq; ++j) {
        const double t = cta_sum(acc[j], red);
        if (threadIdx.x == 0) part[(int64_t(c) * np + i) * nq + j] = t;
    }
    if (threadIdx.x == 0) {
        __threadfence();   // this CTA's partials before its count
        last = atomicAdd(done, 1u) == gridDim.x * gridDim.y * gridDim.z - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // warp per output: lane l adds chunks l, l + 32, ... in order, then the warp tree
    const int lane = threadIdx.x & 31;
    for (int e = threadIdx.x >> 5; e < npq; e += DOT_NT / 32) {
        double s1 = 0.0, s2 = 0.0;
        for (int64_t cc = lane; cc < gridDim.x; cc += 32) s1 += __ldcg(partial + cc * npq + e);
        s1 = warp_sum(s1);
        if (gridDim.z > 1) {
            const double* part2 = partial + int64_t(gridDim.x) * npq;
            for (int64_t cc = lane; cc < gridDim.x; cc += 32) s2 += __ldcg(part2 + cc * npq + e);
            s2 = warp_sum(s2);
        }
        if (lane == 0) {
            out[e] = s1;
            if (gridDim.z > 1) {
                out2[e] = s2;
                if (S) {
                    const int ii = e / nq, jj = e - ii * nq;
                    const double v = 0.5 * (s1 + s2);
                    S[ii * lds + m0 + jj] = v;
                    S[(m0 + jj) * lds + ii] = v;
                }
            }
        }
    }
    if (threadIdx.x == 0) *done = 0u;
}

// Ritz vectors and residuals of the lowest kb pairs in one pass over the vectors:
// X_j = sum_{i<m} U[i][j] V_i, R_j = sum_{i<m} U[i][j] W_i - theta_j X_j (the sums in
// the order of i), and |R_j|^2: per-CTA tree sums in partial, added in a fixed order by the
// CTA that finishes last, which also copies theta_all[0:m] next to them.  kb (at most
// MAXQ pairs per launch; U, theta, X, R and norms point at the launch's first pair) is a
// template parameter (exact loop counts, as for k_multidot).
template <int kb>
__global__ void __launch_bounds__(DOT_NT) k_ritz(const double* __restrict__ U, int ldu, int m,
                                                 const double* __restrict__ V, const double* __restrict__ W,
                                                 int64_t dim, double* __restrict__ X, double* __restrict__ R,
                                                 const double* __restrict__ theta, double* __restrict__ norms,
                                                 const double* __restrict__ theta_all, double* __restrict__ theta_out,
                                                 double* __restrict__ partial, unsigned* __restrict__ done) {
    __shared__ double red[DOT_NT / 32];
    __shared__ bool last;
    double sq[kb];
#pragma unroll
    for (int j = 0; j < kb; ++j) sq[j] = 0.0;
    for (int64_t n = int64_t(blockIdx.x) * DOT_NT + threadIdx.x; n < dim; n += int64_t(gridDim.x) * DOT_NT) {
        double ax[kb], aw[kb];
#pragma unroll
        for (int j = 0; j < kb; ++j) ax[j] = aw[j] = 0.0;
        for (int i = 0; i < m; ++i) {
            const double v = V[i * dim + n], w = W[i * dim + n];
#pragma unroll
            for (int j = 0; j < kb; ++j) {
                const double u = U[i * ldu + j];
                ax[j] += u * v;
                aw[j] += u * w;
            }
        }
#pragma unroll
        for (int j = 0; j < kb; ++j) {
            const double r = aw[j] - theta[j] * ax[j];
            X[j * dim + n] = ax[j];
            R[j * dim + n] = r;
            sq[j] += r * r;
        }
    }
#pragma unroll
    for (int j = 0; j < kb; ++j) {
        const double t = cta_sum(sq[j], red);
        if (threadIdx.x == 0) partial[int64_t(blockIdx.x) * kb + j] = t;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int lane = threadIdx.x & 31;
    for (int j = threadIdx.x >> 5; j < kb; j += DOT_NT / 32) {   // warp per pair, as in k_multidot
        double s = 0.0;
        for (int64_t cc = lane; cc < gridDim.x; cc += 32) s += __ldcg(partial + cc * kb + j);
        s = warp_sum(s);
        if (lane == 0) norms[j] = s;
    }
    for (int j = threadIdx.x; j < m; j += DOT_NT) theta_out[j] = theta_all[j];
    if (threadIdx.x == 0) *done = 0u;
}

// out_j = sum_{i<m} coef[i*ldc + col0 + j] * V_i  (j < nj <= MAXQ); sub: out_j -= ...
// (nj a template parameter, as for k_multidot)
template <int nj>
__global__ void k_lincomb(const double* __restrict__ coef, int ldc, int col0, int m,
                          const double* __restrict__ V, int64_t ldv, int64_t dim, double* __restrict__ out,
                          int64_t ldo, int sub) {
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= dim) return;
    double acc[nj];
#pragma unroll
    for (int j = 0; j < nj; ++j) acc[j] = 0.0;
    for (int i = 0; i < m; ++i) {
        const double v = V[i * ldv + n];
#pragma unroll
        for (int j = 0; j < nj; ++j) acc[j] += coef[i * ldc + col0 + j] * v;
    }
#pragma unroll
    for (int j = 0; j < nj; ++j) {
        if (sub) out[j * ldo + n] -= acc[j];
        else out[j * ldo + n] = acc[j];
    }
}

// Launch of a kernel templated on a vector count 1..MAXQ: LAUNCH(N) is expanded with the
// count as a compile-time constant.
#define DMRG_DISPATCH_COUNT(n, LAUNCH) \
    switch (n) {                      \
        case 1: LAUNCH(1); break;     \
        case 2: LAUNCH(2); break;     \
        case 3: LAUNCH(3); break;     \
        case 4: LAUNCH(4); break;     \
        case 5: LAUNCH(5); break;     \
        case 6: LAUNCH(6); break;     \
        case 7: LAUNCH(7); break;     \
        case 8: LAUNCH(8); break;     \
        default: break;               \
    }

// out = r / (diag - theta[j]) with the denominator floor
__global__ void k_precond(double* __restrict__ out, const double* __restrict__ r, const double* __restrict__ diag,
                          const double* __restrict__ theta, int j, int64_t dim) {
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= dim) return;
    double den = diag[n] - theta[j];
    if (fabs(den) < 1e-8) den = den < 0.0 ? -1e-8 : 1e-8;
    out[n] = r[n] / den;
}

// dst = src / ||src|| with the squared norm read from device memory (zero stays zero)
__global__ void k_normalise(double* __restrict__ dst, const double* __restrict__ src, const double* __restrict__ sq,
                            int64_t dim) {
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const double q = *sq;
    if (n < dim) dst[n] = q > 0.0 ? src[n] / sqrt(q) : 0.0;
}

// Lanczos three-term step: w -= alpha_j q_j + beta_{j-1} q_{j-1} (beta from its square;
// q_prev null for j = 0)
__global__ void k_lanczos_step(double* __restrict__ w, const double* __restrict__ q, const double* __restrict__ q_prev,
                               const double* __restrict__ alpha_j, const double* __restrict__ beta2_prev, int64_t dim) {
    const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= dim) return;
    double v = w[n] - *alpha_j * q[n];
    if (q_prev) v -= sqrt(*beta2_prev) * q_prev[n];
    w[n] = v;
}

// Number of eigenvalues below x of the symmetric tridiagonal matrix with diagonal a[0:n]
// and squared off-diagonal b2[0:n-1]: the sign changes of the characteristic-polynomial
// sequence p_{-1} = 1, p_i(x) = (a_i - x) p_{i-1} - b2_{i-1} p_{i-2} (a zero takes the
// sign opposite to its predecessor; b2 = 0 restarts the sequence).  Division-free: three
// FP64 operations per step (FP64 division is a long chain on this GPU); (p_i, p_{i-1})
// are rescaled by 2^-+256 when their larger exponent leaves [2^-256, 2^256].
__device__ int tri_sturm_count(const double* a, const double* b2, int n, double x) {
    double pp = 1.0, p = a[0] - x;
    int sp = 1, cnt = 0;
    for (int i = 0;; ++i) {
        const long long bits = __double_as_longlong(p);
        const int s = (bits & 0x7FFFFFFFFFFFFFFFll) == 0 ? -sp : (bits < 0 ? -1 : 1);
        cnt += s != sp;
        sp = s;
        if (i + 1 == n) break;
        const int e = max(int((bits >> 52) & 0x7FF), int((__double_as_longlong(pp) >> 52) & 0x7FF));
        if (e > 1023 + 256) {
            p *= 0x1p-256;
            pp *= 0x1p-256;
        } else if (e < 1023 - 256) {
            p *= 0x1p256;
            pp *= 0x1p256;
        }
        const double q = b2[i];
        const double np = q == 0.0 ? (a[i + 1] - x) : fma(-q, pp, (a[i + 1] - x) * p);
        pp = q == 0.0 ? 1.0 : p;
        if (q == 0.0) sp = 1;   // a new block: its sequence starts from p_{-1} = 1
        p = np;
    }
    return cnt;
}

constexpr int TRI_NT = 128;   // multisection points per round (one warp per SM sub-partition)

// Lowest eigenpair of the symmetric tridiagonal T_n (diagonal alpha[0:n], squared
// off-diagonal beta2[0:n-1]) for the Rayleigh-Ritz step of Lanczos, which needs only
// that pair: theta[0] = lambda_min, U[i*ldu] = component i of its unit eigenvector (the
// other columns of U are not touched), and probe = (lambda_min, its last component,
// *beta2_j) for the step's read-back.
// lambda_min by multisection on Sturm counts: the bracket (Gershgorin, widened by a few
// ulps) is cut at TRI_NT points per round, each thread counting the eigenvalues below
// its point, and shrinks to the interval between the last point with none and the first
// with one, until its width is 4 ulps of the matrix scale.  The eigenvector by two steps
// of inverse iteration with the LDL^T factorisation of T - lambda I (pivots kept at least
// one ulp of the scale away from zero), from the all-ones vector.
__global__ void __launch_bounds__(TRI_NT) k_tridiag_lowest(const double* __restrict__ alpha,
                                                          const double* __restrict__ beta2, int n,
                                                          double* __restrict__ theta, double* __restrict__ U, int ldu,
                                                          double* __restrict__ probe,
                                                          const double* __restrict__ beta2_j) {
    __shared__ double a[MAX_BASIS], b2[MAX_BASIS], bb[MAX_BASIS], rd[MAX_BASIS], ll[MAX_BASIS], y[MAX_BASIS];
    __shared__ double red_lo[TRI_NT / 32], red_hi[TRI_NT / 32];
    __shared__ int s_first;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < n; i += TRI_NT) {
        a[i] = alpha[i];
        const double q = i + 1 < n ? beta2[i] : 0.0;
        b2[i] = q;
        bb[i] = sqrt(q);
    }
    __syncthreads();
    // Gershgorin bracket
    double glo = HUGE_VAL, ghi = -HUGE_VAL;
    for (int i = tid; i < n; i += TRI_NT) {
        const double r = (i > 0 ? bb[i - 1] : 0.0) + bb[i];
        glo = fmin(glo, a[i] - r);
        ghi = fmax(ghi, a[i] + r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
        ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    }
    if (lane == 0) {
        red_lo[warp] = glo;
        red_hi[warp] = ghi;
    }
    __syncthreads();
    double lo = red_lo[0], hi = red_hi[0];
    for (int w = 1; w < TRI_NT / 32; ++w) {
        lo = fmin(lo, red_lo[w]);
        hi = fmax(hi, red_hi[w]);
    }
    const double scale = fmax(fabs(lo), fabs(hi));
    const double eps = 0x1p-52;
    lo -= 4.0 * eps * scale + 0x1p-1000;
    hi += 4.0 * eps * scale + 0x1p-1000;
    // multisection: every thread holds the same bracket (the same arithmetic)
    for (int round = 0; round < 24; ++round) {
        const double w = hi - lo;
        if (!(w > 4.0 * eps * scale)) break;
        const double x = lo + w * (double(tid + 1) / double(TRI_NT + 1));
        const int cnt = tri_sturm_count(a, b2, n, x);
        if (tid == 0) s_first = TRI_NT;
        __syncthreads();
        if (cnt >= 1) atomicMin(&s_first, tid);
        __syncthreads();
        const int k = s_first;
        const double nlo = k == 0 ? lo : lo + w * (double(k) / double(TRI_NT + 1));
        const double nhi = k == TRI_NT ? hi : lo + w * (double(k + 1) / double(TRI_NT + 1));
        __syncthreads();   // s_first is read by every thread before the next round resets it
        if (nlo == lo && nhi == hi) break;
        lo = nlo;
        hi = nhi;
    }
    const double lambda = 0.5 * (lo + hi);
    if (tid == 0) {
        // T - lambda I = L D L^T: d_i = (a_i - lambda) - l_{i-1} b_{i-1}, l_i = b_i / d_i
        const double piv = eps * scale + 0x1p-1000;
        double d = a[0] - lambda;
        for (int i = 0; i < n; ++i) {
            if (i > 0) d = (a[i] - lambda) - ll[i - 1] * bb[i - 1];
            if (fabs(d) < piv) d = d < 0.0 ? -piv : piv;
            rd[i] = 1.0 / d;
            ll[i] = bb[i] * rd[i];
        }
        for (int i = 0; i < n; ++i) y[i] = 1.0;
        for (int iter = 0; iter < 2; ++iter) {
            for (int i = 1; i < n; ++i) y[i] -= ll[i - 1] * y[i - 1];   // L z = y
            for (int i = 0; i < n; ++i) y[i] *= rd[i];                  // D w = z
            for (int i = n - 2; i >= 0; --i) y[i] -= ll[i] * y[i + 1];  // L^T x = w
            double mx = 0.0;
            for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(y[i]));
            const double inv = mx > 0.0 ? 1.0 / mx : 1.0;
            double ss = 0.0;
            for (int i = 0; i < n; ++i) {
                y[i] *= inv;
                ss += y[i] * y[i];
            }
            const double r = 1.0 / sqrt(ss);
            for (int i = 0; i < n; ++i) y[i] *= r;
        }
        theta[0] = lambda;
        probe[0] = lambda;
        probe[1] = y[n - 1];
        probe[2] = *beta2_j;
    }
    __syncthreads();
    for (int i = tid; i < n; i += TRI_NT) U[i * ldu] = y[i];
}


// S after a thick restart: diag(theta[0:r]) in the leading r x r block, zero elsewhere
__global__ void k_diag_set(double* __restrict__ S, int lds, int mmax, const double* __restrict__ theta, int r) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mmax * mmax) return;
    const int i = e / mmax, j = e % mmax;
    S[i * lds + j] = (i == j && i < r) ? theta[i] : 0.0;
}

// Integer key whose order is the order of the finite double x.
__device__ __forceinline__ long long order_key(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFll);
}

// Cyclic Jacobi eigensolver of the symmetric m x m matrix S (row stride lds) in one CTA:
// round-robin (circle-method) ordering, the m/2 disjoint rotations of a round applied
// together.  theta ascending, U[i*ldu + j] = component i of eigenvector j.
// Warm start: on entry U[0:mp, 0:mp] (mp < m, or mp = 0 for none) holds the eigenvectors
// of S[0:mp, 0:mp] from the previous call (the Davidson basis only grew since), so the
// sweeps start from B^T S B, B = diag(U[0:mp, 0:mp], I), with the rotations accumulated
// onto B: only the new rows and columns need to be annihilated.
__global__ void __launch_bounds__(256) k_jacobi(const double* __restrict__ S, int m, int lds,
                                                double* __restrict__ theta, double* __restrict__ U, int ldu,
                                                int mp) {
    extern __shared__ double sm[];
    const int M = (m + 1) & ~1;          // even size; a padded index stays decoupled
    const int ld = MAX_BASIS + 1;
    double* A = sm;                      // M x ld
    double* Z = sm + MAX_BASIS * ld;     // eigenvectors, M x ld
    // rotations of a round (compacted), in two sets: the eigenvector update Z <- Z J of a
    // round runs during the next round's angle computation, which occupies one warp
    __shared__ double cs[2][MAX_BASIS / 2], sn[2][MAX_BASIS / 2];
    __shared__ int pp[2][MAX_BASIS / 2], qq[2][MAX_BASIS / 2];
    __shared__ int s_nr[2];
    __shared__ int order[MAX_BASIS];
    const int tid = threadIdx.x, nt = blockDim.x;
    // Z = B;  A = S B (into A), then A = B^T A
    for (int e = tid; e < M * M; e += nt) {
        const int i = e / M, j = e % M;
        Z[i * ld + j] = (i < mp && j < mp) ? U[i * ldu + j] : (i == j ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int e = tid; e < M * M; e += nt) {
        const int i = e / M, j = e % M;
        double v = 0.0;
        if (i < m && j < m) {
            if (j < mp)
                for (int k = 0; k < mp; ++k) v += S[i * lds + k] * Z[k * ld + j];
            else
                v = S[i * lds + j];
        }
        A[i * ld + j] = v;
    }
    __syncthreads();
    double bt[(MAX_BASIS * MAX_BASIS + 255) / 256];   // this thread's entries of B^T A (256 threads)
    int nb = 0;
    for (int e = tid; e < M * M; e += nt) {
        const int i = e / M, j = e % M;
        double v = A[i * ld + j];
        if (i < mp) {
            v = 0.0;
            for (int k = 0; k < mp; ++k) v += Z[k * ld + i] * A[k * ld + j];
        }
        bt[nb++] = v;
    }
    __syncthreads();
    nb = 0;
    for (int e = tid; e < M * M; e += nt) {
        const int i = e / M, j = e % M;
        A[i * ld + j] = bt[nb++];
    }
    __syncthreads();
    const int half = M / 2;   // <= 32: the angles of a round are computed by warp 0
    __shared__ int s_rot;
    // Z <- Z J for the n rotations of set b, by threads t0, t0 + step, ...
    auto z_update = [&](int b, int n, int t0, int step) {
        for (int e = t0; e < n * M; e += step) {
            const int k = e / M, row = e % M;
            const int p = pp[b][k], q = qq[b][k];
            const double c = cs[b][k], s = sn[b][k];
            const double u = Z[row * ld + p], w = Z[row * ld + q];
            Z[row * ld + p] = c * u - s * w;
            Z[row * ld + q] = s * u + c * w;
        }
    };
    if (tid == 0) s_nr[0] = s_nr[1] = 0;
    int cur = 0;              // set of this round's rotations
    int pend = 0, pend_n = 0; // set and count of the rotations not yet applied to Z
    __syncthreads();
    for (int sweep = 0; sweep < 40 && M >= 2; ++sweep) {
        // converged when no pair passes the rotation test (the sweep would rotate nothing):
        // one pass over the matrix instead of a sweep of rounds
        int any = 0;
        for (int e = tid; e < M * M; e += nt) {
            const int i = e / M, j = e % M;
            if (i < j && jacobi_rotate_needed(A[i * ld + j], A[i * ld + i], A[j * ld + j])) any = 1;
        }
        if (!__syncthreads_or(any)) break;
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int r = 0; r < M - 1; ++r) {
            // s_nr[cur] is zero here
            if (tid < half) {
                const int k = tid;
                const int a = k == 0 ? 0 : ((k - 1 + r) % (M - 1)) + 1;
                const int b = ((M - 2 - k + r) % (M - 1)) + 1;
                const int p = min(a, b), q = max(a, b);
                const double apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
                // rotate only while the off-diagonal entry is above rounding level
                if (jacobi_rotate_needed(apq, app, aqq)) {
                    double c, s;
                    jacobi_rotation(aqq - app, apq, &c, &s);
                    const int slot = atomicAdd(&s_nr[cur], 1);
                    pp[cur][slot] = p; qq[cur][slot] = q; cs[cur][slot] = c; sn[cur][slot] = s;
                    s_rot = 1;
                }
            } else if (tid >= 32) {
                z_update(pend, pend_n, tid - 32, nt - 32);   // the previous round's rotations
            }
            __syncthreads();
            // the disjoint rotations of this round, in any order; every thread reads the
            // same count.  The other set's Z update has finished: its count is cleared for
            // the next round (no thread reads it before the next barrier)
            const int nr = s_nr[cur];
            pend = cur;
            pend_n = nr;
            if (tid == 0) s_nr[cur ^ 1] = 0;
            cur ^= 1;
            if (nr == 0) {
                __syncthreads();
                continue;
            }
            for (int e = tid; e < nr * M; e += nt) {       // A <- A J
                const int k = e / M, row = e % M;
                const int p = pp[pend][k], q = qq[pend][k];
                const double c = cs[pend][k], s = sn[pend][k];
                const double x = A[row * ld + p], y = A[row * ld + q];
                A[row * ld + p] = c * x - s * y;
                A[row * ld + q] = s * x + c * y;
            }
            __syncthreads();
            for (int e = tid; e < nr * M; e += nt) {       // A <- J^T A
                const int k = e / M, col = e % M;
                const int p = pp[pend][k], q = qq[pend][k];
                const double c = cs[pend][k], s = sn[pend][k];
                const double x = A[p * ld + col], y = A[q * ld + col];
                A[p * ld + col] = c * x - s * y;
                A[q * ld + col] = s * x + c * y;
            }
            __syncthreads();
        }
        if (s_rot == 0) break;   // a sweep without rotations: converged to rounding level
        __syncthreads();
    }
    z_update(pend, pend_n, tid, nt);   // the last round's rotations
    __syncthreads();
    // ascending order of the m real eigenvalues (ties by index): the rank of eigenvalue
    // i is the count of those before it, compared as integers (order-preserving keys)
    for (int i = tid; i < m; i += nt) {
        const long long ki = order_key(A[i * ld + i]);
        int rank = 0;
        for (int j = 0; j < m; ++j) {
            const long long kj = order_key(A[j * ld + j]);
            rank += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
        }
        order[rank] = i;
    }
    __syncthreads();
    for (int j = tid; j < m; j += nt) theta[j] = A[order[j] * ld + order[j]];
    for (int e = tid; e < m * m; e += nt) {
        const int i = e / m, j = e % m;
        U[i * ldu + j] = Z[i * ld + order[j]];
    }
}

inline unsigned blocks_for(int64_t n, int t = 256) { return unsigned((n + t - 1) / t); }

}  // namespace

void Handle::release_davidson() {
    delete dav;
    dav = nullptr;
}

namespace {

struct Run {
    Handle* h;
    DavidsonState* s;
    int64_t dim;
    int mmax;
    cudaStream_t st = nullptr;

    int check(cudaError_t e, const char* what) { return e == cudaSuccess ? DMRG_OK : cuda_fail(e, what); }

    // out[i*nq + j] = P_i . Q_j  (np <= MAX_BASIS, nq <= MAXQ); result in s->small
    int dots(const double* P, int np, const double* Q, int nq, double* out) {
        if (np == 0 || nq == 0) return DMRG_OK;
#define DMRG_DOTS(N)                                                                                      \
    k_multidot<N><<<dim3(unsigned(s->n_chunks), unsigned(np)), DOT_NT, 0, st>>>(                          \
        P, dim, np, Q, dim, dim, s->chunk, s->partial, out, s->done, nullptr, nullptr, nullptr, nullptr, 0, 0)
        DMRG_DISPATCH_COUNT(nq, DMRG_DOTS)
#undef DMRG_DOTS
        return check(cudaGetLastError(), "dot kernel");
    }
    int lincomb(const double* coef, int ldc, int col0, int nj, int m, const double* V, double* out, int sub) {
        for (int j0 = 0; j0 < nj; j0 += MAXQ) {
            const int n = nj - j0 < MAXQ ? nj - j0 : MAXQ;
#define DMRG_LINCOMB(N)                                                                                   \
    k_lincomb<N><<<blocks_for(dim), 256, 0, st>>>(coef, ldc, col0 + j0, m, V, dim, dim, out + j0 * dim, dim, sub)
            DMRG_DISPATCH_COUNT(n, DMRG_LINCOMB)
#undef DMRG_LINCOMB
        }
        return check(cudaGetLastError(), "lincomb");
    }
    // CGS2 of v against V[0:m]; appends it as V[m] when kept.  Both norms stay on the
    // device (the normalisation reads the second); one read-back decides whether the
    // vector is kept (norm after CGS2 >= 1e-10 of the norm before).
    int cgs2_append(double* v, int* m, bool* kept) {
        *kept = false;
        double* nrm = s->small;   // [0] = |v|^2 before, [1] = after
        int rc = dots(v, 1, v, 1, nrm);
        if (rc) return rc;
        for (int pass = 0; pass < 2; ++pass) {
            if (*m == 0) break;
            double* d = s->small + 64;
            for (int i0 = 0; i0 < *m; i0 += MAX_BASIS) {
                const int ni = *m - i0 < MAX_BASIS ? *m - i0 : MAX_BASIS;
                if ((rc = dots(s->V + i0 * dim, ni, v, 1, d + i0))) return rc;
            }
            k_lincomb<1><<<blocks_for(dim), 256, 0, st>>>(d, 1, 0, *m, s->V, dim, dim, v, dim, 1);
            if ((rc = check(cudaGetLastError(), "cgs update"))) return rc;
        }
        if ((rc = dots(v, 1, v, 1, nrm + 1))) return rc;
        k_normalise<<<blocks_for(dim), 256, 0, st>>>(s->V + int64_t(*m) * dim, v, nrm + 1, dim);
        if ((rc = check(cudaGetLastError(), "normalise"))) return rc;
        double n2[2];
        if ((rc = check(cudaMemcpy(n2, nrm, sizeof(n2), cudaMemcpyDeviceToHost), "read norms"))) return rc;
        const double n0 = std::sqrt(n2[0]), n1 = std::sqrt(n2[1]);
        if (!(n0 > 0.0) || n1 < 1e-10 * n0) return DMRG_OK;   // V[m] is left to be overwritten
        *m += 1;
        *kept = true;
        return DMRG_OK;
    }
    // S entries of the new columns [m0, m): S_ij = (V_i.W_j + V_j.W_i)/2, both dot sets and
    // the update in one launch
    int s_update(int m0, int m) {
        const int nb = m - m0;
        double* g1 = s->small + 256;
        double* g2 = g1 + MAX_BASIS * MAXQ;
        for (int j0 = 0; j0 < nb; j0 += MAXQ) {
            const int nq = nb - j0 < MAXQ ? nb - j0 : MAXQ;
#define DMRG_SUPD(N)                                                                                          \
    k_multidot<N><<<dim3(unsigned(s->n_chunks), unsigned(m), 2u), DOT_NT, 0, st>>>(                           \
        s->V, dim, m, s->W + int64_t(m0 + j0) * dim, dim, dim, s->chunk, s->partial, g1, s->done, s->W,        \
        s->V + int64_t(m0 + j0) * dim, g2, s->S, mmax, m0 + j0)
            DMRG_DISPATCH_COUNT(nq, DMRG_SUPD)
#undef DMRG_SUPD
            int rc;
            if ((rc = check(cudaGetLastError(), "S update"))) return rc;
        }
        return DMRG_OK;
    }
    // Ritz vectors X, residuals R and |R_j|^2 (into small[2048 + j]) with theta[0:m] next to
    // them (small[2048 + MAX_BASIS + j]), one launch
    int ritz(int kb, int m) {
        const int64_t grid = std::min<int64_t>((dim + DOT_NT - 1) / DOT_NT, s->n_chunks * MAX_BASIS);
        for (int j0 = 0; j0 < kb; j0 += MAXQ) {   // MAXQ pairs per launch
            const int n = kb - j0 < MAXQ ? kb - j0 : MAXQ;
#define DMRG_RITZ(N)                                                                                       \
    k_ritz<N><<<unsigned(grid), DOT_NT, 0, st>>>(s->U + j0, mmax, m, s->V, s->W, dim, s->X + j0 * dim,       \
                                                 s->R + j0 * dim, s->theta + j0, s->small + 2048 + j0, s->theta, \
                                                 s->small + 2048 + MAX_BASIS, s->partial, s->done)
            DMRG_DISPATCH_COUNT(n, DMRG_RITZ)
#undef DMRG_RITZ
        }
        return check(cudaGetLastError(), "ritz vectors");
    }
};

}  // namespace
}  // namespace dmrg

namespace dmrg {
namespace {

// The solver buffers of a handle, kept between calls of the same shape.
int ensure_state(Handle* h, int mmax, int kbmax, int block, int k_eig) {
    if (h->dav && (h->dav->mmax != mmax || h->dav->kbmax != kbmax || h->dav->block != block ||
                   h->dav->k_eig != k_eig))
        h->release_davidson();
    if (h->dav) return DMRG_OK;
    const int64_t dim = h->plan.dim;
    h->dav = new DavidsonState();
    DavidsonState* s = h->dav;
    const int64_t want = 2 * int64_t(h->n_sm);
    s->chunk = std::max<int64_t>(DOT_MIN_CHUNK, (dim + want - 1) / want);
    s->chunk = (s->chunk + DOT_NT - 1) / DOT_NT * DOT_NT;
    s->n_chunks = (dim + s->chunk - 1) / s->chunk;
    s->mmax = mmax; s->kbmax = kbmax; s->block = block; s->k_eig = k_eig;
    auto al = [&](double** p, int64_t n, const char* w) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(double) * (n > 0 ? n : 1));
        return e == cudaSuccess ? DMRG_OK : cuda_fail(e, w);
    };
    int rc;
    if ((rc = al(&s->V, int64_t(mmax) * dim, "V")) || (rc = al(&s->W, int64_t(mmax) * dim, "W")) ||
        (rc = al(&s->X, int64_t(kbmax) * dim, "X")) || (rc = al(&s->R, int64_t(kbmax) * dim, "R")) ||
        (rc = al(&s->C, int64_t(block) * dim, "C")) || (rc = al(&s->T, int64_t(k_eig + block) * dim, "T")) ||
        (rc = al(&s->diag, dim, "diag")) || (rc = al(&s->S, mmax * mmax, "S")) ||
        (rc = al(&s->U, mmax * mmax, "U")) || (rc = al(&s->theta, mmax, "theta")) ||
        (rc = al(&s->small, 4096, "small")) || (rc = al(&s->partial, 2 * s->n_chunks * MAX_BASIS * MAXQ, "partials"))) {
        h->release_davidson();
        return rc;
    }
    cudaError_t ce = cudaMalloc(reinterpret_cast<void**>(&s->done), sizeof(unsigned));
    if (ce == cudaSuccess) ce = cudaMemset(s->done, 0, sizeof(unsigned));
    if (ce != cudaSuccess) {
        h->release_davidson();
        return cuda_fail(ce, "dot counter");
    }
    cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(sizeof(double) * 2 * MAX_BASIS * (MAX_BASIS + 1)));
    return DMRG_OK;
}

}  // namespace
}  // namespace dmrg

using dmrg::Handle;

extern "C" int dmrg_davidson(dmrg_heff_t hh, int32_t k_eig, double tol, int32_t max_iter, int32_t block,
                             int32_t n_iter, double* x_inout, double* evals, dmrg_davidson_info* info) {
    using namespace dmrg;
    const auto t_start = std::chrono::steady_clock::now();
    if (!hh) return fail(DMRG_ERR_INVALID_ARG, "null handle");
    Handle* h = static_cast<Handle*>(hh);
    if (h->plan_only) return fail(DMRG_ERR_INVALID_ARG, "plan-only handle");
    const int64_t dim = h->plan.dim;
    if (k_eig < 1 || block < 1 || block > MAXQ || block > h->max_nvec || max_iter < 1 || n_iter < 0 ||
        !(tol >= 0.0))
        return fail(DMRG_ERR_INVALID_ARG, "k_eig >= 1, 1 <= block <= min(8, max_nvec), max_iter >= 1, tol >= 0");
    const int mmax = 8 * block > 24 ? 8 * block : 24;
    if (mmax < k_eig + 2 * block || mmax > MAX_BASIS) return fail(DMRG_ERR_INVALID_ARG, "k_eig too large for the basis");
    if (dim < int64_t(k_eig) + block) return fail(DMRG_ERR_INVALID_ARG, "problem smaller than k_eig + block");
    if (!x_inout || !evals) return fail(DMRG_ERR_INVALID_ARG, "null x_inout or evals");

    const int kbmax = k_eig > block ? k_eig : block;
    int rc;
    if ((rc = ensure_state(h, mmax, kbmax, block, k_eig))) return rc;
    const size_t jac_smem = sizeof(double) * 2 * MAX_BASIS * (MAX_BASIS + 1);
    cudaStream_t st = nullptr;
    DavidsonState* s = h->dav;
    Run run{h, s, dim, mmax};
    if (!s->diag_ready) {
        if ((rc = h->diagonal(s->diag, st))) return rc;
        s->diag_ready = true;
    }

    // start block
    int m = 0;
    bool kept;
    if ((rc = run.check(cudaMemcpy(s->C, x_inout, sizeof(double) * block * dim, cudaMemcpyDeviceToDevice), "x0")))
        return rc;
    for (int j = 0; j < block; ++j)
        if ((rc = run.cgs2_append(s->C + j * dim, &m, &kept))) return rc;
    if (m == 0) return fail(DMRG_ERR_INVALID_ARG, "start block is numerically zero");
    if ((rc = h->apply(s->V, s->W, m, st))) return rc;
    int matvecs = m, restarts = 0;
    if ((rc = run.s_update(0, m))) return rc;

    std::vector<double> th(mmax), rn(mmax), rb(size_t(2 * MAX_BASIS));
    int it = 0, kb = 0;
    int m_prev = 0;   // rows of U that diagonalise S[0:m_prev, 0:m_prev] (warm start)
    bool converged = false;
    while (it < max_iter) {
        ++it;
        k_jacobi<<<1, 256, jac_smem, st>>>(s->S, m, mmax, s->theta, s->U, mmax, m_prev < m ? m_prev : 0);
        if ((rc = run.check(cudaGetLastError(), "jacobi"))) return rc;
        m_prev = m;
        kb = m < kbmax ? m : kbmax;
        if ((rc = run.ritz(kb, m))) return rc;
        // Ritz values next to the residual norms: one read-back per step
        if ((rc = run.check(cudaMemcpy(rb.data(), s->small + 2048, sizeof(double) * (MAX_BASIS + m),
                                       cudaMemcpyDeviceToHost),
                            "read residuals and theta")))
            return rc;
        for (int j = 0; j < kb; ++j) rn[j] = rb[size_t(j)];
        for (int j = 0; j < m; ++j) th[j] = rb[size_t(MAX_BASIS + j)];
        for (int j = 0; j < kb; ++j) rn[j] = std::sqrt(rn[j]);
        if (info && info->hist_theta && it <= info->hist_cap) info->hist_theta[it - 1] = th[0];
        if (info && info->hist_time && it <= info->hist_cap)
            info->hist_time[it - 1] =
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        bool all = kb >= k_eig;
        for (int j = 0; j < k_eig && j < kb; ++j) all = all && rn[j] <= tol;
        if (all) {
            converged = true;
            break;
        }
        if (n_iter > 0 && it >= n_iter) break;
        std::vector<int> sel;
        for (int j = 0; j < kb && int(sel.size()) < block; ++j)
            if (rn[j] > tol) sel.push_back(j);
        for (size_t c = 0; c < sel.size(); ++c)
            k_precond<<<blocks_for(dim), 256, 0, st>>>(s->C + c * dim, s->R + sel[c] * dim, s->diag, s->theta, sel[c],
                                                       dim);
        if (m + int(sel.size()) > mmax) {   // thick restart
            const int r = m < k_eig + block ? m : k_eig + block;
            if ((rc = run.lincomb(s->U, mmax, 0, r, m, s->V, s->T, 0))) return rc;
            if ((rc = run.check(cudaMemcpy(s->V, s->T, sizeof(double) * r * dim, cudaMemcpyDeviceToDevice), "V restart")))
                return rc;
            if ((rc = run.lincomb(s->U, mmax, 0, r, m, s->W, s->T, 0))) return rc;
            if ((rc = run.check(cudaMemcpy(s->W, s->T, sizeof(double) * r * dim, cudaMemcpyDeviceToDevice), "W restart")))
                return rc;
            k_diag_set<<<blocks_for(mmax * mmax), 256, 0, st>>>(s->S, mmax, mmax, s->theta, r);
            m = r;
            m_prev = 0;   // the rotated basis: S[0:r, 0:r] is diagonal
            ++restarts;
        }
        const int m_old = m;
        for (size_t c = 0; c < sel.size(); ++c)
            if ((rc = run.cgs2_append(s->C + c * dim, &m, &kept))) return rc;
        if (m == m_old) break;
        if ((rc = h->apply(s->V + int64_t(m_old) * dim, s->W + int64_t(m_old) * dim, m - m_old, st))) return rc;
        matvecs += m - m_old;
        if ((rc = run.s_update(m_old, m))) return rc;
    }
    const int k = k_eig < kb ? k_eig : kb;
    if ((rc = run.check(cudaMemcpy(x_inout, s->X, sizeof(double) * k * dim, cudaMemcpyDeviceToDevice), "x out"))) return rc;
    if ((rc = run.check(cudaDeviceSynchronize(), "davidson"))) return rc;
    if ((rc = h->check_status())) return rc;
    double rmax = 0.0;
    for (int j = 0; j < k; ++j) {
        evals[j] = th[j];
        rmax = rn[j] > rmax ? rn[j] : rmax;
    }
    if (info) {
        info->iters = it;
        info->matvecs = matvecs;
        info->converged = converged ? 1 : 0;
        info->restarts = restarts;
        info->resid_max = rmax;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    }
    return converged || n_iter > 0 ? DMRG_OK : DMRG_ERR_NOT_CONVERGED;
}

// Lowest eigenpair by restarted Lanczos with full reorthogonalisation (the steps are
// listed with the oracle's variant): per step one apply, alpha_j, the three-term step,
// two Gram-Schmidt passes against the basis, beta_j, and Rayleigh-Ritz on the growing
// tridiagonal T (its lowest pair only, k_tridiag_lowest); one read-back per step.
extern "C" int dmrg_lanczos(dmrg_heff_t hh, double tol, int32_t max_iter, int32_t m_max, double* x_inout,
                            double* eval, dmrg_davidson_info* info) {
    using namespace dmrg;
    const auto t_start = std::chrono::steady_clock::now();
    if (!hh) return fail(DMRG_ERR_INVALID_ARG, "null handle");
    Handle* h = static_cast<Handle*>(hh);
    if (h->plan_only) return fail(DMRG_ERR_INVALID_ARG, "plan-only handle");
    const int64_t dim = h->plan.dim;
    if (max_iter < 1 || m_max < 2 || m_max > MAX_BASIS - 1 || !(tol >= 0.0))
        return fail(DMRG_ERR_INVALID_ARG, "max_iter >= 1, 2 <= m_max <= 63, tol >= 0");
    if (dim < 2) return fail(DMRG_ERR_INVALID_ARG, "problem smaller than 2");
    if (!x_inout || !eval) return fail(DMRG_ERR_INVALID_ARG, "null x_inout or eval");
    const int mmax = m_max + 1;   // the basis holds q_0 .. q_{m_max}
    int rc;
    if ((rc = ensure_state(h, mmax, 1, 1, 1))) return rc;
    DavidsonState* s = h->dav;
    cudaStream_t st = nullptr;
    Run run{h, s, dim, mmax};
    double* alpha = s->small + 3000;   // alpha_j (device)
    double* beta2 = s->small + 3100;   // beta_j^2 (device)
    double* probe = s->small + 3200;
    // q_0 = x0 / ||x0||
    if ((rc = run.check(cudaMemcpy(s->R, x_inout, sizeof(double) * dim, cudaMemcpyDeviceToDevice), "x0"))) return rc;
    int m = 0;
    bool kept = false;
    if ((rc = run.cgs2_append(s->R, &m, &kept))) return rc;
    if (!kept) return fail(DMRG_ERR_INVALID_ARG, "start vector is numerically zero");
    int it = 0, matvecs = 0, restarts = 0, n = 0;
    double theta = 0.0;
    bool converged = false, restart = false;
    while (it < max_iter) {
        if (restart) {   // T has m_max rows: restart from the Ritz vector y = sum_i s_i q_i
            if ((rc = run.lincomb(s->U, mmax, 0, 1, n, s->V, s->C, 0))) return rc;
            m = 0;
            if ((rc = run.cgs2_append(s->C, &m, &kept))) return rc;
            if (!kept) return fail(DMRG_ERR_INVALID_ARG, "Ritz vector is numerically zero");
            ++restarts;
            restart = false;
        }
        ++it;
        const int j = m - 1;   // the newest basis vector q_j
        const double* qj = s->V + int64_t(j) * dim;
        if ((rc = h->apply(qj, s->R, 1, st))) return rc;
        ++matvecs;
        if ((rc = run.dots(qj, 1, s->R, 1, alpha + j))) return rc;
        k_lanczos_step<<<blocks_for(dim), 256, 0, st>>>(s->R, qj, j > 0 ? qj - dim : nullptr, alpha + j,
                                                        beta2 + (j > 0 ? j - 1 : 0), dim);
        if ((rc = run.check(cudaGetLastError(), "lanczos step"))) return rc;
        // full reorthogonalisation; q_{j+1} appended when w did not vanish
        if ((rc = run.cgs2_append(s->R, &m, &kept))) return rc;
        if ((rc = run.check(cudaMemcpyAsync(beta2 + j, s->small + 1, sizeof(double), cudaMemcpyDeviceToDevice, st),
                            "beta")))
            return rc;
        n = j + 1;   // T_j is n x n
        k_tridiag_lowest<<<1, TRI_NT, 0, st>>>(alpha, beta2, n, s->theta, s->U, mmax, probe, beta2 + j);
        if ((rc = run.check(cudaGetLastError(), "lanczos ritz"))) return rc;
        double pr[3];
        if ((rc = run.check(cudaMemcpy(pr, probe, sizeof(pr), cudaMemcpyDeviceToHost), "read ritz"))) return rc;
        theta = pr[0];
        if (info && info->hist_theta && it <= info->hist_cap) info->hist_theta[it - 1] = theta;
        if (info && info->hist_time && it <= info->hist_cap)
            info->hist_time[it - 1] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if (std::sqrt(pr[2]) * std::fabs(pr[1]) <= tol || !kept) {   // converged, or invariant Krylov space
            converged = true;
            break;
        }
        restart = n == m_max;
    }
    // Ritz vector of the last T (n x n), normalised, and its explicit residual
    if ((rc = run.lincomb(s->U, mmax, 0, 1, n, s->V, s->C, 0))) return rc;
    int m1 = 0;
    if ((rc = run.cgs2_append(s->C, &m1, &kept))) return rc;   // V[0] = y / ||y||
    if (!kept) return fail(DMRG_ERR_INVALID_ARG, "Ritz vector is numerically zero");
    if ((rc = h->apply(s->V, s->R, 1, st))) return rc;
    ++matvecs;
    if ((rc = run.check(cudaMemcpy(x_inout, s->V, sizeof(double) * dim, cudaMemcpyDeviceToDevice), "x out"))) return rc;
    k_lanczos_step<<<blocks_for(dim), 256, 0, st>>>(s->R, s->V, nullptr, s->theta, nullptr, dim);   // H y - theta y
    double r2 = 0.0;
    if ((rc = run.dots(s->R, 1, s->R, 1, s->small + 3300))) return rc;
    if ((rc = run.check(cudaMemcpy(&r2, s->small + 3300, sizeof(double), cudaMemcpyDeviceToHost), "residual"))) return rc;
    if ((rc = run.check(cudaDeviceSynchronize(), "lanczos"))) return rc;
    if ((rc = h->check_status())) return rc;
    *eval = theta;
    if (info) {
        info->iters = it;
        info->matvecs = matvecs;
        info->converged = converged ? 1 : 0;
        info->restarts = restarts;
        info->resid_max = std::sqrt(r2);
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    }
    return converged ? DMRG_OK : DMRG_ERR_NOT_CONVERGED;
}
