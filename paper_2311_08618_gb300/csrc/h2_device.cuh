// Device helpers shared by the construction and factorization kernels:
// kernel entries, the sketch generator and CTA-cooperative dense routines
// (Householder QR with column pivoting, Bunch-Kaufman LDL^T) in FP64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace h2dev {

// --------------------------------------------------------------- kernels --
struct KernelSpec {
    int kind;
    double p0, p1, p2, p3;
};

// A_ij = f(|x_i - x_j|) for the kernels of Sec. 5 (see h2_kernel_kind).
__device__ __forceinline__ double kernel_entry(const KernelSpec& k, const double* xi,
                                               const double* xj) {
    double dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    switch (k.kind) {
        case 0: return 1.0 / (r + k.p0);
        case 1: return exp(-r) / (r + k.p0);
        case 2: return exp(-0.5 * r * r) + k.p0 / (r + k.p1);
        case 3: return r < 0.5 ? 2.0 : (fabs(r - 1.0) < 0.5 ? -1.0 : 0.0);
        default: return fmin(xi[0], xj[0]);
    }
}

// SplitMix64 (Vigna; Steele, Lea & Flood 2014): output number `idx` (0-based)
// of the generator started at state `seed`.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t idx) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (idx + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Sketch entry Omega[i][c] = (2u - 1) * scale, u = top 53 bits * 2^-53.
__device__ __forceinline__ double sketch_entry(uint64_t seed, int64_t i, int c, int s,
                                               double scale) {
    uint64_t z = splitmix64_at(seed, (uint64_t)i * (uint64_t)s + (uint64_t)c);
    double u = (double)(z >> 11) * 0x1.0p-53;
    return (2.0 * u - 1.0) * scale;
}

// ------------------------------------------------------- block reductions --
template <int NT>
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < NT / 32 ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    double r = red[0];
    __syncthreads();
    return r;
}

// argmax with the first index on ties; returns index, writes value
template <int NT>
__device__ int block_argmax(double v, int idx, double* redv, int* redi, double* outv) {
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) { redv[w] = v; redi[w] = idx; }
    __syncthreads();
    if (w == 0) {
        v = lane < NT / 32 ? redv[lane] : -1.0;
        idx = lane < NT / 32 ? redi[lane] : 0x7fffffff;
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, v, o);
            int oi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
        }
        if (lane == 0) { redv[0] = v; redi[0] = idx; }
    }
    __syncthreads();
    int r = redi[0];
    *outv = redv[0];
    __syncthreads();
    return r;
}

// argmax (first index on ties) with a single barrier: warp-shuffle
// reduction, one partial per warp in shared memory, then every thread reduces
// the partials itself.  `buf` alternates between two halves (par selects the
// half) so that consecutive calls need no trailing barrier: a thread can only
// reach call n+2 (same half) after every thread passed the barrier of call n+1,
// i.e. after every thread finished reading the partials of call n.
template <int NT>
__device__ __forceinline__ int block_argmax1(double v, int idx, double* bufv, int* bufi, int par,
                                             double* outv) {
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    const int w = threadIdx.x >> 5;
    double* bv = bufv + par * (NT / 32);
    int* bi = bufi + par * (NT / 32);
    if ((threadIdx.x & 31) == 0) { bv[w] = v; bi[w] = idx; }
    __syncthreads();
    v = bv[0];
    idx = bi[0];
#pragma unroll
    for (int u = 1; u < NT / 32; ++u) {
        double ov = bv[u];
        int oi = bi[u];
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    *outv = v;
    return idx;
}

// sum with a single barrier, double-buffered like block_argmax1 (the partials
// of the warps are added in warp order, the same on every thread)
template <int NT>
__device__ __forceinline__ double block_sum1(double v, double* buf, int par) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    double* b = buf + par * (NT / 32);
    if ((threadIdx.x & 31) == 0) b[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = b[0];
#pragma unroll
    for (int u = 1; u < NT / 32; ++u) r += b[u];
    return r;
}

// Ordering key of |x|: the bit pattern of a non-negative double, read as an
// unsigned integer, orders like its value (a NaN ranks above +inf).  Pivot
// searches compare these keys in the integer pipes.
__device__ __forceinline__ unsigned long long abs_key(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Block argmax of (key, index): the largest key, the smallest index on ties,
// the same on every thread.  Within a warp three integer reductions (high
// word, low word among the maxima, index among the exact maxima); across
// warps one barrier and a scan of the warps' winners.  bk / bi: 2 * NTH / 32
// entries each, double-buffered by par like block_argmax1.
template <int NTH>
__device__ __forceinline__ int block_argmax_key(unsigned long long key, int idx, unsigned long long* bk, int* bi,
                                                int par, unsigned long long* out_key) {
    constexpr int NW = NTH / 32;
    const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
    const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    const unsigned mi = __reduce_min_sync(0xffffffffu, (hi == mh && lo == ml) ? (unsigned)idx : 0xffffffffu);
    unsigned long long* k2 = bk + par * NW;
    int* i2 = bi + par * NW;
    if ((threadIdx.x & 31) == 0) {
        k2[threadIdx.x >> 5] = ((unsigned long long)mh << 32) | ml;
        i2[threadIdx.x >> 5] = (int)min(mi, 0x7fffffffu);
    }
    __syncthreads();
    unsigned long long kb = k2[0];
    int ib = i2[0];
#pragma unroll
    for (int u = 1; u < NW; ++u) {
        const unsigned long long ku = k2[u];
        const int iu = i2[u];
        if (ku > kb || (ku == kb && iu < ib)) { kb = ku; ib = iu; }
    }
    *out_key = kb;
    return ib;
}

// ------------------------------------------------- pivoted Householder QR --
// Householder QR with column pivoting of Y (m x s, row-major, leading
// dimension ldy), in place, stopped when the Frobenius norm of the
// not-yet-pivoted remainder Y[k:, k:] is <= tol, or after `cap` steps.
// Reflector k is stored in V (row-major m x ldv, column k, rows k..m-1,
// unit 2-norm; a zero vector means H_k = I).  Returns k (the rank).  All
// threads of the CTA call it.
//
// The column norms of step k+1 are recomputed exactly (no downdating), in the
// same pass that applies reflector k: the sum over rows k+1..m-1 of the
// updated column, in row order.  The pivot column k itself is not updated (it
// is never read again: only the reflectors are used).  Pivot: the largest
// norm, the smallest column index among equal norms.
template <int NT>
__device__ int cta_pivqr(double* Y, int ldy, int m, int s, double tol, int cap, double* V,
                         int ldv, double* red, int* redi, int* bad = nullptr) {
    // red / redi: at least 2 * NT / 32 entries (double-buffered reductions)
    int kmax = min(min(m, s), cap);
    int k = 0;
    int par = 0;
    double part = 0.0, best = -1.0;
    int bi = 0x7fffffff;
    for (int j = threadIdx.x; j < s; j += NT) {        // norms of step 0
        double a = 0.0;
        for (int i = 0; i < m; ++i) {
            double y = Y[(size_t)i * ldy + j];
            a += y * y;
        }
        part += a;
        if (a > best) { best = a; bi = j; }
    }
    for (; k < kmax; ++k) {
        double total = block_sum1<NT>(part, red, par);
        par ^= 1;
        if (!(total == total)) {          // NaN input: stop, report, touch nothing
            if (bad && threadIdx.x == 0) *bad = 1;
            break;
        }
        if (total <= tol * tol) break;
        // pivot: the largest norm (integer keys of the non-negative norms,
        // smallest index on ties), no FP64 compare on the step's chain
        unsigned long long bk;
        const bool has = bi != 0x7fffffff;
        int jp = block_argmax_key<NT>(has ? abs_key(best) : 0ull, has ? bi : 0x7fffffff,
                                      reinterpret_cast<unsigned long long*>(red), redi, par, &bk);
        par ^= 1;
        if (jp < k || jp >= s) jp = k;
        if (jp != k)
            for (int i = threadIdx.x; i < m; i += NT) {
                double t = Y[(size_t)i * ldy + k];
                Y[(size_t)i * ldy + k] = Y[(size_t)i * ldy + jp];
                Y[(size_t)i * ldy + jp] = t;
            }
        __syncthreads();
        // reflector from x = Y[k:, k]; |x|^2 is the pivot column's norm that
        // won the search (summed over rows k.. in the previous update)
        const double nx2 = __longlong_as_double((long long)bk);
        double nx = sqrt(nx2);
        double x0 = Y[(size_t)k * ldy + k];
        double alpha = x0 >= 0.0 ? -nx : nx;
        // |v|^2 = |x|^2 - 2 alpha x0 + alpha^2 = 2 |x|^2 + 2 |x0| |x| (alpha has
        // the opposite sign of x0, so nothing cancels): no second reduction
        double v0 = x0 - alpha;
        double nv = sqrt(2.0 * nx2 + 2.0 * fabs(x0) * nx);
        const double inv_nv = nv > 0.0 ? 1.0 / nv : 0.0;
        for (int i = threadIdx.x; i < m; i += NT) {
            double x = 0.0;
            if (i >= k && nv > 0.0) x = ((i == k) ? v0 : Y[(size_t)i * ldy + k]) * inv_nv;
            V[(size_t)i * ldv + k] = x;
        }
        __syncthreads();
        // Y[k:, j] -= 2 v (v . Y[k:, j]) for j > k, and the norms of step k+1
        part = 0.0;
        best = -1.0;
        bi = 0x7fffffff;
        for (int j = k + 1 + threadIdx.x; j < s; j += NT) {
            double a = 0.0;
            if (nv > 0.0) {
                double w = 0.0;
                for (int i = k; i < m; ++i) w += V[(size_t)i * ldv + k] * Y[(size_t)i * ldy + j];
                w *= 2.0;
                Y[(size_t)k * ldy + j] -= w * V[(size_t)k * ldv + k];
                for (int i = k + 1; i < m; ++i) {
                    double y = Y[(size_t)i * ldy + j] - w * V[(size_t)i * ldv + k];
                    Y[(size_t)i * ldy + j] = y;
                    a += y * y;
                }
            } else {
                for (int i = k + 1; i < m; ++i) {
                    double y = Y[(size_t)i * ldy + j];
                    a += y * y;
                }
            }
            part += a;
            if (a > best) { best = a; bi = j; }
        }
        __syncthreads();
    }
    __syncthreads();
    return k;
}

// Q = H_0 H_1 ... H_{k-1} (m x m, row-major, leading dimension ldq) from the
// reflectors stored by cta_pivqr, applied to the identity from the last one
// back.  H_r changes only rows and columns r.. of the product, so reflector
// r is the (m - r) x (m - r) update Q[r:, r:] -= 2 v (v^T Q[r:, r:]).  Its
// dot products are split into P = NT / (m - r) row chunks per column (the
// partials are added in chunk order), so that each thread's chain of
// dependent FP64 operations is short; the update spreads the entries over
// all threads.  All threads of the CTA call it.
template <int NT>
__device__ void cta_form_q(double* Q, int ldq, int m, const double* V, int ldv, int k) {
    __shared__ double fq[2 * NT];
    for (int e = threadIdx.x; e < m * m; e += NT) {
        int i = e / m, j = e % m;
        Q[(size_t)i * ldq + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int r = k - 1; r >= 0; --r) {
        const int c = m - r;     // columns and rows r.. of the update
        const double* v = V + (size_t)r * ldv + r;   // v_i = v[(i - r) * ldv]
        if (c > 2 * NT) {
            for (int j = r + threadIdx.x; j < m; j += NT) {
                double w = 0.0;
                for (int i = r; i < m; ++i) w += V[(size_t)i * ldv + r] * Q[(size_t)i * ldq + j];
                w *= 2.0;
                if (w != 0.0)
                    for (int i = r; i < m; ++i) Q[(size_t)i * ldq + j] -= w * V[(size_t)i * ldv + r];
            }
            __syncthreads();
            continue;
        }
        const int P = c <= NT ? NT / c : 1;
        const int len = (c + P - 1) / P;
        double* wv = P > 1 ? fq + NT : fq;         // 2 v^T Q[r:, j], j = r + jj
        for (int t = threadIdx.x; t < P * c; t += NT) {
            const int jj = t % c, ch = t / c;
            const int i0 = ch * len, i1 = min(c, i0 + len);
            double w = 0.0;
            for (int ii = i0; ii < i1; ++ii) w += v[(size_t)ii * ldv] * Q[(size_t)(r + ii) * ldq + r + jj];
            if (P > 1) fq[ch * c + jj] = w;
            else wv[jj] = 2.0 * w;
        }
        __syncthreads();
        if (P > 1) {
            for (int jj = threadIdx.x; jj < c; jj += NT) {
                double w = 0.0;
                for (int ch = 0; ch < P; ++ch) w += fq[ch * c + jj];
                wv[jj] = 2.0 * w;
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < c * c; e += NT) {
            const int ii = e / c, jj = e % c;
            Q[(size_t)(r + ii) * ldq + r + jj] -= wv[jj] * v[(size_t)ii * ldv];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------ Bunch-Kaufman LDL --
// In-place Bunch-Kaufman LDL^T (partial pivoting, alpha = (1 + sqrt 17)/8) of
// the full symmetric n x n matrix S (row-major, leading dimension lds).  On
// return the strict lower triangle holds L (except the (k+1, k) entry of a
// 2x2 pivot, which is D's off-diagonal), the diagonal holds D, perm[j] is the
// original index of position j, and piv[j] = 1 (1x1), 2 (first of a 2x2),
// 0 (second of a 2x2).  Accumulates #negative eigenvalues of D into *neg and
// the smallest |eigenvalue| of a D block into *minpiv (thread 0's values).
// buf: 4n doubles (shared memory preferred): the pivot column(s) and the
// multipliers of the current step, so that the trailing update divides once
// per row (l_i = c_i / d) and then only multiplies (S_ij -= l_i c_j).
template <int NT>
__device__ void cta_bk_ldl(double* S, int lds, int n, int* perm, int* piv, double* red,
                           int* redi, int* neg, double* minpiv, int* bad, double zero_pivot,
                           double* buf) {
    // red / redi: at least 2 * NT / 32 entries each (double-buffered argmax)
    const double alpha = (1.0 + sqrt(17.0)) / 8.0;
    constexpr int NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* c0 = buf;
    double* c1 = buf + n;
    double* l0 = buf + 2 * n;
    double* l1 = buf + 3 * n;
    for (int i = threadIdx.x; i < n; i += NT) perm[i] = i;
    __syncthreads();
    int k = 0;
    int nneg = 0;
    int par = 0;
    double mp = 1.0 / 0.0;
    while (k < n) {
        double akk = fabs(S[(size_t)k * lds + k]);
        // lam = max_{i>k} |S_ik|, r = first index attaining it
        double best = -1.0;
        int bi = 0x7fffffff;
        for (int i = k + 1 + threadIdx.x; i < n; i += NT) {
            double v = fabs(S[(size_t)i * lds + k]);
            if (v > best) { best = v; bi = i; }
        }
        double lam;
        int r = block_argmax1<NT>(best, bi, red, redi, par, &lam);
        par ^= 1;
        if (k + 1 >= n) { lam = 0.0; r = k; }
        else if (r <= k || r >= n) r = k + 1;
        int size = 1;
        int swap_a = -1, swap_b = -1;
        if (!(akk == akk) || !(lam == lam)) {
            if (threadIdx.x == 0) *bad = 1;   // NaN: finish with 1x1 steps, flagged
        } else if (!(lam == 0.0 || akk >= alpha * lam)) {
            double b2 = -1.0;
            int bj = 0x7fffffff;
            for (int j = k + threadIdx.x; j < n; j += NT) {
                if (j == r) continue;
                double v = fabs(S[(size_t)j * lds + r]);
                if (v > b2) { b2 = v; bj = j; }
            }
            double sig;
            block_argmax1<NT>(b2, bj, red, redi, par, &sig);
            par ^= 1;
            if (sig < 0.0) sig = 0.0;
            if (akk * sig >= alpha * lam * lam) {
                // 1x1 at k
            } else if (fabs(S[(size_t)r * lds + r]) >= alpha * sig) {
                swap_a = k; swap_b = r;
            } else {
                swap_a = k + 1; swap_b = r;
                size = 2;
            }
        }
        if (swap_a >= 0 && swap_a != swap_b) {
            // swap rows then columns swap_a <-> swap_b (all of them)
            __syncthreads();   // every thread has read S for the pivot search
            for (int j = threadIdx.x; j < n; j += NT) {
                double t = S[(size_t)swap_a * lds + j];
                S[(size_t)swap_a * lds + j] = S[(size_t)swap_b * lds + j];
                S[(size_t)swap_b * lds + j] = t;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += NT) {
                double t = S[(size_t)i * lds + swap_a];
                S[(size_t)i * lds + swap_a] = S[(size_t)i * lds + swap_b];
                S[(size_t)i * lds + swap_b] = t;
            }
            if (threadIdx.x == 0) {
                int t = perm[swap_a];
                perm[swap_a] = perm[swap_b];
                perm[swap_b] = t;
            }
        }
        __syncthreads();
        if (size == 1) {
            double d = S[(size_t)k * lds + k];
            if (d == 0.0 && zero_pivot != 0.0) d = zero_pivot;   // zero column: stored as zero_pivot
            if (threadIdx.x == 0) {
                S[(size_t)k * lds + k] = d;
                piv[k] = 1;
                if (d < 0.0) nneg += 1;
                mp = fmin(mp, fabs(d));
                if (d != d) *bad = 1;
            }
            if (d != 0.0 && k + 1 < n) {
                // c = S[k+1:, k], l = c (1/d) ; S[k+1:, k+1:] -= l c^T ; S[k+1:, k] = l
                const double invd = 1.0 / d;
                for (int i = k + 1 + threadIdx.x; i < n; i += NT) {
                    double c = S[(size_t)i * lds + k];
                    c0[i] = c;
                    l0[i] = c * invd;
                }
                __syncthreads();
                for (int i = k + 1 + warp; i < n; i += NW) {
                    const double li = l0[i];
                    double* Si = S + (size_t)i * lds;
                    for (int j = k + 1 + lane; j < n; j += 32) Si[j] -= li * c0[j];
                }
                for (int i = k + 1 + threadIdx.x; i < n; i += NT) S[(size_t)i * lds + k] = l0[i];
            }
            __syncthreads();
            k += 1;
        } else {
            double a = S[(size_t)k * lds + k], b = S[(size_t)(k + 1) * lds + k],
                   c = S[(size_t)(k + 1) * lds + k + 1];
            double det = a * c - b * b;
            if (threadIdx.x == 0) {
                piv[k] = 2;
                piv[k + 1] = 0;
                double tr = a + c;
                nneg += det < 0.0 ? 1 : (tr < 0.0 ? 2 : 0);
                double disc = sqrt(fmax(0.0, 0.25 * (a - c) * (a - c) + b * b));
                double e0 = 0.5 * tr - disc, e1 = 0.5 * tr + disc;
                mp = fmin(mp, fmin(fabs(e0), fabs(e1)));
                if (det != det) *bad = 1;
            }
            if (k + 2 < n) {
                // Lc = C E^{-1}; S[k+2:, k+2:] -= Lc C^T ; store Lc in S[k+2:, k:k+2]
                const double idet = 1.0 / det;
                double i00 = c * idet, i01 = -b * idet, i11 = a * idet;
                for (int i = k + 2 + threadIdx.x; i < n; i += NT) {
                    double ci0 = S[(size_t)i * lds + k], ci1 = S[(size_t)i * lds + k + 1];
                    c0[i] = ci0;
                    c1[i] = ci1;
                    l0[i] = ci0 * i00 + ci1 * i01;
                    l1[i] = ci0 * i01 + ci1 * i11;
                }
                __syncthreads();
                for (int i = k + 2 + warp; i < n; i += NW) {
                    const double a0 = l0[i], a1 = l1[i];
                    double* Si = S + (size_t)i * lds;
                    for (int j = k + 2 + lane; j < n; j += 32) Si[j] -= a0 * c0[j] + a1 * c1[j];
                }
                for (int i = k + 2 + threadIdx.x; i < n; i += NT) {
                    S[(size_t)i * lds + k] = l0[i];
                    S[(size_t)i * lds + k + 1] = l1[i];
                }
            }
            __syncthreads();
            k += 2;
        }
    }
    if (threadIdx.x == 0) {
        *neg += nneg;
        *minpiv = fmin(*minpiv, mp);
    }
    __syncthreads();
}

// S[i][j] -= a_i b_j (+ a2_i b2_j) over the lower triangle o <= j <= i < n of
// a row-major block.  The rows are taken in folded pairs (o + q, n - 1 - q),
// whose q + 1 and n - o - q entries make one span of n - o + 1 (the middle
// row of an odd count alone); warp w takes spans w, w + NW, ... and its lanes
// walk the span, so every warp gets about the same number of elements.
template <bool TWO, int NW>
__device__ __forceinline__ void lower_rank_update(double* S, int lds, int o, int n, const double* a, const double* b,
                                                  const double* a2, const double* b2) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = n - o;
    const int P = (t + 1) >> 1;
    for (int q = warp; q < P; q += NW) {
        const int ra = o + q, rb = n - 1 - q;
        const int len = ra == rb ? q + 1 : t + 1;
        for (int m = lane; m < len; m += 32) {
            const int i = m <= q ? ra : rb;
            const int j = m <= q ? o + m : o + m - q - 1;
            double v = S[(size_t)i * lds + j];
            if (TWO) v -= a[i] * b[j] + a2[i] * b2[j];
            else v -= a[i] * b[j];
            S[(size_t)i * lds + j] = v;
        }
    }
}

// |x| (given by its key) as a float scaled by 2^(1023 - eref), eref being the
// biased exponent of the largest value it is compared with; the mantissa is
// truncated to 23 bits and values below 2^-126 of the reference read as 0.
// Integer operations only.
__device__ __forceinline__ float key_scaled(unsigned long long key, int eref) {
    const int e = (int)(key >> 52) - eref + 127;
    if (e <= 0) return 0.0f;
    return __uint_as_float(((unsigned)e << 23) | ((unsigned)(key >> 29) & 0x7fffffu));
}

// Bunch-Kaufman LDL^T of an n x n symmetric block on one CTA of NTH threads,
// reading and updating only the lower triangle and diagonal of S (the strict
// upper triangle is neither read nor written).  The output is cta_bk_ldl's
// packed factor (L strictly below the diagonal except the (k + 1, k) entry of
// a 2x2 pivot, which holds D's off-diagonal; D on the diagonal; perm, piv).
//
// On this GPU an FP64 instruction of a warp holds its sub-partition's FP64
// unit for many cycles, and a pivot step is a chain of dependent scalar
// operations, so the FP64 work is kept off that chain where exactness does
// not need it:
//   - the pivot searches compare |values| as integer keys (largest value,
//     first index on ties; a NaN ranks largest and flags *bad);
//   - the test |a_kk| >= alpha lambda (alpha = (1 + sqrt 17) / 8) is made
//     on 24-bit scaled copies of the two values (the threshold moves by at
//     most 2^-23 relative); the tests of a pivoting step (after the search
//     of column r) stay in FP64;
//   - the negative count and the smallest |pivot| are formed after the loop,
//     one pivot block per thread;
//   - the trailing update touches the triangle only (half of cta_bk_ldl's
//     products), balanced across the warps.
// Keep lds odd when S is in shared memory: the column reads of the pivot
// search are then free of bank conflicts.  rk / ri: 2 * NTH / 32 entries
// each; buf: 4n values.  neg / minpiv / bad: thread 0 accumulates.
template <int NTH>
__device__ void cta_bk_ldl_lower(double* S, int lds, int n, int* perm, int* piv, unsigned long long* rk, int* ri,
                                 int* neg, double* minpiv, int* bad, double zero_pivot, double* buf) {
    constexpr int NW = NTH / 32;
    constexpr unsigned long long kInf = 0x7ff0000000000000ull;
    const double alpha = (1.0 + sqrt(17.0)) / 8.0;
    const float alpha_f = 0.640388203f;   // alpha rounded to FP32
    const int tid = threadIdx.x;
    const bool zp = zero_pivot != 0.0;
    double* c0 = buf;
    double* c1 = buf + n;
    double* l0 = buf + 2 * n;
    double* l1 = buf + 3 * n;
    for (int i = tid; i < n; i += NTH) perm[i] = i;
    __syncthreads();
    int k = 0, par = 0, flag_nan = 0;
    while (k < n) {
        const unsigned long long akey = abs_key(S[(size_t)k * lds + k]);
        unsigned long long key = 0;
        int bi = 0x7fffffff;
        for (int i = k + 1 + tid; i < n; i += NTH) {
            const unsigned long long v = abs_key(S[(size_t)i * lds + k]);
            if (v > key) { key = v; bi = i; }
        }
        unsigned long long lk;
        int r = block_argmax_key<NTH>(key, bi, rk, ri, par, &lk);
        par ^= 1;
        if (k + 1 >= n) { lk = 0; r = k; }
        else if (r <= k || r >= n) r = k + 1;
        int size = 1;
        int swap_a = -1, swap_b = -1;
        bool test = false;
        if (akey > kInf || lk > kInf) {
            flag_nan = 1;   // NaN: finish with 1x1 steps, flagged
        } else if (lk != 0) {
            const int eref = (int)(max(akey, lk) >> 52);
            test = !(key_scaled(akey, eref) >= alpha_f * key_scaled(lk, eref));
        }
        if (test) {
            // sig = max_{j >= k, j != r} |S_jr| from the lower triangle
            const double akk = __longlong_as_double((long long)akey), lam = __longlong_as_double((long long)lk);
            const double arr = __longlong_as_double((long long)abs_key(S[(size_t)r * lds + r]));
            key = 0;
            bi = 0x7fffffff;
            for (int j = k + tid; j < n; j += NTH) {
                if (j == r) continue;
                const unsigned long long v = abs_key(j > r ? S[(size_t)j * lds + r] : S[(size_t)r * lds + j]);
                if (v > key) { key = v; bi = j; }
            }
            unsigned long long sk;
            block_argmax_key<NTH>(key, bi, rk, ri, par, &sk);
            par ^= 1;
            const double sig = __longlong_as_double((long long)sk);
            if (akk * sig >= alpha * lam * lam) {
                // 1x1 at k
            } else if (arr >= alpha * sig) {
                swap_a = k; swap_b = r;
            } else {
                swap_a = k + 1; swap_b = r;
                size = 2;
            }
        }
        if (swap_a >= 0 && swap_a != swap_b) {
            // symmetric interchange of sa < sb in lower-triangle storage
            const int sa = swap_a, sb = swap_b;
            __syncthreads();   // every thread has read S for the searches
            for (int j = tid; j < sa; j += NTH) {
                const double t = S[(size_t)sa * lds + j];
                S[(size_t)sa * lds + j] = S[(size_t)sb * lds + j];
                S[(size_t)sb * lds + j] = t;
            }
            for (int i = sa + 1 + tid; i < sb; i += NTH) {
                const double t = S[(size_t)i * lds + sa];
                S[(size_t)i * lds + sa] = S[(size_t)sb * lds + i];
                S[(size_t)sb * lds + i] = t;
            }
            for (int i = sb + 1 + tid; i < n; i += NTH) {
                const double t = S[(size_t)i * lds + sa];
                S[(size_t)i * lds + sa] = S[(size_t)i * lds + sb];
                S[(size_t)i * lds + sb] = t;
            }
            if (tid == 0) {
                const double t = S[(size_t)sa * lds + sa];
                S[(size_t)sa * lds + sa] = S[(size_t)sb * lds + sb];
                S[(size_t)sb * lds + sb] = t;
                const int q = perm[sa];
                perm[sa] = perm[sb];
                perm[sb] = q;
            }
            __syncthreads();
        }
        if (size == 1) {
            double d = S[(size_t)k * lds + k];
            const bool dz = abs_key(d) == 0;
            if (dz && zp) d = zero_pivot;   // zero column: stored as zero_pivot
            const bool elim = !(dz && !zp) && k + 1 < n;
            if (elim) {
                const double invd = 1.0 / d;
                for (int i = k + 1 + tid; i < n; i += NTH) {
                    const double c = S[(size_t)i * lds + k];
                    const double l = c * invd;
                    c0[i] = c;
                    l0[i] = l;
                    S[(size_t)i * lds + k] = l;
                }
            }
            __syncthreads();
            if (tid == 0) {
                S[(size_t)k * lds + k] = d;
                piv[k] = 1;
            }
            if (elim) {
                lower_rank_update<false, NW>(S, lds, k + 1, n, l0, c0, nullptr, nullptr);
                __syncthreads();
            }
            k += 1;
        } else {
            const double a = S[(size_t)k * lds + k], b = S[(size_t)(k + 1) * lds + k],
                         c = S[(size_t)(k + 1) * lds + k + 1];
            if (k + 2 < n) {
                const double det = a * c - b * b;
                const double idet = 1.0 / det;
                const double i00 = c * idet, i01 = -b * idet, i11 = a * idet;
                for (int i = k + 2 + tid; i < n; i += NTH) {
                    const double ci0 = S[(size_t)i * lds + k], ci1 = S[(size_t)i * lds + k + 1];
                    const double a0 = ci0 * i00 + ci1 * i01, a1 = ci0 * i01 + ci1 * i11;
                    c0[i] = ci0;
                    c1[i] = ci1;
                    l0[i] = a0;
                    l1[i] = a1;
                    S[(size_t)i * lds + k] = a0;
                    S[(size_t)i * lds + k + 1] = a1;
                }
            }
            __syncthreads();
            if (tid == 0) {
                piv[k] = 2;
                piv[k + 1] = 0;
            }
            if (k + 2 < n) {
                lower_rank_update<true, NW>(S, lds, k + 2, n, l0, c0, l1, c1);
                __syncthreads();
            }
            k += 2;
        }
    }
    __syncthreads();
    // the inertia of D and its smallest |eigenvalue|, one pivot block per
    // thread: a 1x1 pivot d counts if d < 0; a 2x2 block [a b; b c] has one
    // negative eigenvalue if det < 0, two if det >= 0 and a + c < 0
    int nn = 0, nb = 0;
    unsigned long long mk = kInf;
    for (int j = tid; j < n; j += NTH) {
        const int pv = piv[j];
        if (pv == 1) {
            const double d = S[(size_t)j * lds + j];
            const unsigned long long dk = abs_key(d);
            nn += (__double_as_longlong(d) < 0 && dk != 0 && dk <= kInf) ? 1 : 0;
            if (dk > kInf) nb = 1;
            mk = min(mk, dk);
        } else if (pv == 2) {
            const double a = S[(size_t)j * lds + j], b = S[(size_t)(j + 1) * lds + j],
                         c = S[(size_t)(j + 1) * lds + j + 1];
            const double det = a * c - b * b, tr = a + c;
            nn += det < 0.0 ? 1 : (tr < 0.0 ? 2 : 0);
            const double disc = sqrt(fmax(0.0, 0.25 * (a - c) * (a - c) + b * b));
            const double e0 = 0.5 * tr - disc, e1 = 0.5 * tr + disc;
            mk = min(mk, min(abs_key(e0), abs_key(e1)));
            if (det != det) nb = 1;
        }
    }
    nn = __reduce_add_sync(0xffffffffu, nn);
    nb = __reduce_or_sync(0xffffffffu, nb);
    {
        const unsigned hi = (unsigned)(mk >> 32), lo = (unsigned)mk;
        const unsigned mh = __reduce_min_sync(0xffffffffu, hi);
        const unsigned ml = __reduce_min_sync(0xffffffffu, hi == mh ? lo : 0xffffffffu);
        mk = ((unsigned long long)mh << 32) | ml;
    }
    unsigned long long* k2 = rk + par * NW;
    int* i2 = ri + par * NW;
    if ((tid & 31) == 0) {
        k2[tid >> 5] = mk;
        i2[tid >> 5] = nn | (nb << 30);
    }
    __syncthreads();
    if (tid == 0) {
        int tn = 0, tb = flag_nan;
        unsigned long long tm = kInf;
        for (int u = 0; u < NW; ++u) {
            tn += i2[u] & 0x3fffffff;
            tb |= i2[u] >> 30;
            tm = min(tm, k2[u]);
        }
        *neg += tn;
        *minpiv = fmin(*minpiv, __longlong_as_double((long long)tm));
        if (tb) *bad = 1;
    }
    __syncthreads();
}

// argmax over a warp: the largest v, the smallest index on ties
__device__ __forceinline__ void warp_argmax(double& v, int& idx) {
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
}

// Trailing update of one Bunch-Kaufman step on a warp:
//   S[o + i][o + j] -= a[o + i] * b[o + j]                        (1x1 pivot)
//   S[o + i][o + j] -= a[o + i] * b[o + j] + a2[o + i] * b2[o + j]  (2x2 pivot)
// for i, j < t.  The lanes walk the flattened t x t block 32 elements apart
// (di rows and dj columns per step); each lane loads four elements before it
// stores any, so their products overlap in the FP64 pipe.
template <bool TWO>
__device__ __forceinline__ void warp_trailing_update(double* S, int lds, int o, int t, const double* a,
                                                     const double* b, const double* a2, const double* b2) {
    const int lane = threadIdx.x & 31;
    const int di = 32 / t, dj = 32 % t;
    int i = lane / t, j = lane % t;
    int e = lane;
    for (; e + 96 < t * t; e += 128) {
        int ii[4], jj[4];
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            ii[u] = o + i;
            jj[u] = o + j;
            i += di;
            j += dj;
            if (j >= t) { j -= t; ++i; }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = S[(size_t)ii[u] * lds + jj[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (TWO) v[u] -= a[ii[u]] * b[jj[u]] + a2[ii[u]] * b2[jj[u]];
            else v[u] -= a[ii[u]] * b[jj[u]];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) S[(size_t)ii[u] * lds + jj[u]] = v[u];
    }
    for (; e < t * t; e += 32) {
        const int ig = o + i, jg = o + j;
        if (TWO) S[(size_t)ig * lds + jg] -= a[ig] * b[jg] + a2[ig] * b2[jg];
        else S[(size_t)ig * lds + jg] -= a[ig] * b[jg];
        i += di;
        j += dj;
        if (j >= t) { j -= t; ++i; }
    }
}

// The same Bunch-Kaufman LDL^T as cta_bk_ldl, run by one warp: the same
// pivot search (largest |value|, first index on ties), the same decisions and
// the same expression for every updated element, with warp shuffles for the
// reductions and __syncwarp for the barriers.  The trailing update walks the
// (row, column) pairs of the trailing block as one flat index, so no lane
// idles on a partial row (warp_trailing_update).  neg / minpiv / bad are
// lane 0's accumulators.
__device__ inline void warp_bk_ldl(double* S, int lds, int n, int* perm, int* piv, int* neg, double* minpiv, int* bad,
                            double zero_pivot, double* buf) {
    const double alpha = (1.0 + sqrt(17.0)) / 8.0;
    const int lane = threadIdx.x & 31;
    double* c0 = buf;
    double* c1 = buf + n;
    double* l0 = buf + 2 * n;
    double* l1 = buf + 3 * n;
    for (int i = lane; i < n; i += 32) perm[i] = i;
    __syncwarp();
    int k = 0, nneg = 0;
    double mp = 1.0 / 0.0;
    while (k < n) {
        double akk = fabs(S[(size_t)k * lds + k]);
        double lam = -1.0;
        int r = 0x7fffffff;
        for (int i = k + 1 + lane; i < n; i += 32) {
            double v = fabs(S[(size_t)i * lds + k]);
            if (v > lam) { lam = v; r = i; }
        }
        warp_argmax(lam, r);
        if (k + 1 >= n) { lam = 0.0; r = k; }
        else if (r <= k || r >= n) r = k + 1;
        int size = 1;
        int swap_a = -1, swap_b = -1;
        if (!(akk == akk) || !(lam == lam)) {
            if (lane == 0) *bad = 1;
        } else if (!(lam == 0.0 || akk >= alpha * lam)) {
            double sig = -1.0;
            int bj = 0x7fffffff;
            for (int j = k + lane; j < n; j += 32) {
                if (j == r) continue;
                double v = fabs(S[(size_t)j * lds + r]);
                if (v > sig) { sig = v; bj = j; }
            }
            warp_argmax(sig, bj);
            if (sig < 0.0) sig = 0.0;
            if (akk * sig >= alpha * lam * lam) {
                // 1x1 at k
            } else if (fabs(S[(size_t)r * lds + r]) >= alpha * sig) {
                swap_a = k; swap_b = r;
            } else {
                swap_a = k + 1; swap_b = r;
                size = 2;
            }
        }
        if (swap_a >= 0 && swap_a != swap_b) {
            __syncwarp();
            for (int j = lane; j < n; j += 32) {
                double t = S[(size_t)swap_a * lds + j];
                S[(size_t)swap_a * lds + j] = S[(size_t)swap_b * lds + j];
                S[(size_t)swap_b * lds + j] = t;
            }
            __syncwarp();
            for (int i = lane; i < n; i += 32) {
                double t = S[(size_t)i * lds + swap_a];
                S[(size_t)i * lds + swap_a] = S[(size_t)i * lds + swap_b];
                S[(size_t)i * lds + swap_b] = t;
            }
            if (lane == 0) {
                int t = perm[swap_a];
                perm[swap_a] = perm[swap_b];
                perm[swap_b] = t;
            }
        }
        __syncwarp();
        if (size == 1) {
            double d = S[(size_t)k * lds + k];
            if (d == 0.0 && zero_pivot != 0.0) d = zero_pivot;
            __syncwarp();
            if (lane == 0) {
                S[(size_t)k * lds + k] = d;
                piv[k] = 1;
                if (d < 0.0) nneg += 1;
                mp = fmin(mp, fabs(d));
                if (d != d) *bad = 1;
            }
            const int t = n - k - 1;
            if (d != 0.0 && t > 0) {
                const double invd = 1.0 / d;
                for (int i = k + 1 + lane; i < n; i += 32) {
                    double c = S[(size_t)i * lds + k];
                    c0[i] = c;
                    l0[i] = c * invd;
                }
                __syncwarp();
                warp_trailing_update<false>(S, lds, k + 1, t, l0, c0, nullptr, nullptr);
                for (int i = k + 1 + lane; i < n; i += 32) S[(size_t)i * lds + k] = l0[i];
            }
            __syncwarp();
            k += 1;
        } else {
            double a = S[(size_t)k * lds + k], b = S[(size_t)(k + 1) * lds + k],
                   c = S[(size_t)(k + 1) * lds + k + 1];
            double det = a * c - b * b;
            if (lane == 0) {
                piv[k] = 2;
                piv[k + 1] = 0;
                double tr = a + c;
                nneg += det < 0.0 ? 1 : (tr < 0.0 ? 2 : 0);
                double disc = sqrt(fmax(0.0, 0.25 * (a - c) * (a - c) + b * b));
                double e0 = 0.5 * tr - disc, e1 = 0.5 * tr + disc;
                mp = fmin(mp, fmin(fabs(e0), fabs(e1)));
                if (det != det) *bad = 1;
            }
            const int t = n - k - 2;
            if (t > 0) {
                const double idet = 1.0 / det;
                double i00 = c * idet, i01 = -b * idet, i11 = a * idet;
                for (int i = k + 2 + lane; i < n; i += 32) {
                    double ci0 = S[(size_t)i * lds + k], ci1 = S[(size_t)i * lds + k + 1];
                    c0[i] = ci0;
                    c1[i] = ci1;
                    l0[i] = ci0 * i00 + ci1 * i01;
                    l1[i] = ci0 * i01 + ci1 * i11;
                }
                __syncwarp();
                warp_trailing_update<true>(S, lds, k + 2, t, l0, c0, l1, c1);
                for (int i = k + 2 + lane; i < n; i += 32) {
                    S[(size_t)i * lds + k] = l0[i];
                    S[(size_t)i * lds + k + 1] = l1[i];
                }
            }
            __syncwarp();
            k += 2;
        }
    }
    if (lane == 0) {
        *neg += nneg;
        *minpiv = fmin(*minpiv, mp);
    }
    __syncwarp();
}

// L(j, i) of the unit lower factor stored by cta_bk_ldl (i < j).
__device__ __forceinline__ double bk_L(const double* S, int lds, const int* piv, int j, int i) {
    if (piv[i] == 2 && j == i + 1) return 0.0;
    return S[(size_t)j * lds + i];
}

}  // namespace h2dev
