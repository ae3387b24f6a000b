// H^2 construction on the device (Sec. 3.1): nested orthogonal shared bases
// from a rank-revealing (column-pivoted Householder) QR of the sketched far row
// A_{l;c,+} Omega (Eqs. shared-bases and transfer-matrices), skeleton couplings
// S^SS = U_c^S^T A_cd U_d^S of far pairs (Eq. lr_skeleton) and transformed
// leaf near blocks [U^S U^R]^T A_cd [U^S U^R] (Eq. dense_skeleton).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "h2_device.cuh"
#include "h2_internal.h"

using namespace h2dev;

namespace h2 {

#define CK(x)                                                                       \
    do {                                                                            \
        cudaError_t e_ = (x);                                                       \
        if (e_ != cudaSuccess) {                                                    \
            set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x); \
            return e_ == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA;      \
        }                                                                           \
    } while (0)

template <typename T>
static int dalloc(T** p, size_t count) {
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return H2_ERR_OOM;
    }
    return H2_OK;
}

template <typename T>
static int upload(T** p, const std::vector<T>& v) {
    int rc = dalloc(p, v.size());
    if (rc) return rc;
    if (!v.empty()) CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return H2_OK;
}

// ---------------------------------------------------------------- kernels --
constexpr int NT = 256;

// row absolute sums and diagonal of A (exact, O(n^2) evaluations)
__global__ void k_rowsum(KernelSpec ks, const double* __restrict__ X, int64_t n,
                         double* rowabs, double* diag) {
    int64_t i = blockIdx.x;
    __shared__ double red[32];
    const double* xi = X + 3 * i;
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += NT) acc += fabs(kernel_entry(ks, xi, X + 3 * j));
    acc = block_sum<NT>(acc, red);
    if (threadIdx.x == 0) {
        rowabs[i] = acc;
        diag[i] = kernel_entry(ks, xi, xi);
    }
}

// out[0] = max rowabs, out[1] = min(A_ii - R_i), out[2] = max(A_ii + R_i)
__global__ void k_gershgorin(const double* rowabs, const double* diag, int64_t n, double* out) {
    __shared__ double smax[NT], smin[NT], shi[NT];
    double mx = 0.0, lo = 1.0 / 0.0, hi = -1.0 / 0.0;
    for (int64_t i = threadIdx.x; i < n; i += NT) {
        double R = rowabs[i] - fabs(diag[i]);
        mx = fmax(mx, rowabs[i]);
        lo = fmin(lo, diag[i] - R);
        hi = fmax(hi, diag[i] + R);
    }
    smax[threadIdx.x] = mx; smin[threadIdx.x] = lo; shi[threadIdx.x] = hi;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
            shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = smax[0]; out[1] = smin[0]; out[2] = shi[0]; }
}

__global__ void k_omega(double* Om, int64_t n, int s, uint64_t seed, double scale) {
    int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= n * s) return;
    Om[e] = sketch_entry(seed, e / s, (int)(e % s), s, scale);
}

// Z[tau][h] (m x s) = sum over leaves sigma with h(tau,sigma) = h of A(tau,sigma) Omega(sigma)
// grid: (entry of the (tau,h) work list); CSR of sigma leaves per entry.
// A work item is (row i, group of CPT sketch columns): each kernel entry is
// evaluated once per group and reused for the group's columns.
constexpr int CPT = 16;
__global__ void k_sketch(KernelSpec ks, const double* __restrict__ X, const double* __restrict__ Om,
                         int s, const int64_t* __restrict__ leaf_off, const int* __restrict__ wl_tau,
                         const int* __restrict__ wl_h, const int* __restrict__ wl_ptr,
                         const int* __restrict__ wl_sigma, int L, int mmax, double* Z) {
    int w = blockIdx.x;
    int tau = wl_tau[w], h = wl_h[w];
    int64_t r0 = leaf_off[tau];
    int m = (int)(leaf_off[tau + 1] - r0);
    int groups = (s + CPT - 1) / CPT;
    double* Zt = Z + ((size_t)tau * L + h) * (size_t)mmax * s;
    for (int e = threadIdx.x; e < m * groups; e += NT) {
        int i = e % m, g = e / m;
        int c0 = g * CPT;
        const double* xi = X + 3 * (r0 + i);
        double acc[CPT];
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) acc[cc] = 0.0;
        for (int q = wl_ptr[w]; q < wl_ptr[w + 1]; ++q) {
            int sg = wl_sigma[q];
            for (int64_t j = leaf_off[sg]; j < leaf_off[sg + 1]; ++j) {
                double a = kernel_entry(ks, xi, X + 3 * j);
                const double* om = Om + j * s + c0;
#pragma unroll
                for (int cc = 0; cc < CPT; ++cc)
                    if (c0 + cc < s) acc[cc] += a * om[cc];
            }
        }
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc)
            if (c0 + cc < s) Zt[(size_t)i * s + c0 + cc] = acc[cc];
    }
}

// Y_l restricted to leaf tau rows = sum_{h < l} Z[tau][h]; written into the
// level's row-space buffer Ylev (n x s, tree order)
__global__ void k_sum_levels(const double* Z, const int64_t* leaf_off, int L, int mmax, int s,
                             int l, double* Ylev) {
    int tau = blockIdx.x;
    int64_t r0 = leaf_off[tau];
    int m = (int)(leaf_off[tau + 1] - r0);
    for (int e = threadIdx.x; e < m * s; e += NT) {
        double acc = 0.0;
        for (int h = 0; h < l; ++h) acc += Z[((size_t)tau * L + h) * (size_t)mmax * s + e];
        Ylev[(size_t)r0 * s + e] = acc;
    }
}

// Leaf bases: pivoted QR of Y_L(tau) (m x s) -> Q_tau (m x m), rank; E rows.
// Upper bases: Yhat = [E_c1^T Y(c1 rows); E_c2^T Y(c2 rows)] -> T_P.
// grid: clusters of the level.  scratch per cluster: Yhat (dq x s), V (dq x dq).
__global__ void k_basis(const double* Ylev, int s, const int64_t* off, int leaf_level,
                        const double* Echild, int rbc, const int* rb_child, int dq, double tol,
                        int cap, double* scratch, double* Qout, int* rank_out, double* resid_out) {
    int c = blockIdx.x;
    __shared__ double red[32];
    __shared__ int redi[32];
    double* Yh = scratch + (size_t)c * ((size_t)dq * s + (size_t)dq * dq);
    double* V = Yh + (size_t)dq * s;
    int64_t r0 = off[c];
    int m;
    if (leaf_level) {
        m = (int)(off[c + 1] - r0);
        for (int e = threadIdx.x; e < m * s; e += NT) Yh[e] = Ylev[(size_t)r0 * s + e];
    } else {
        int c1 = 2 * c, c2 = 2 * c + 1;
        int r1 = rb_child[c1], r2 = rb_child[c2];
        m = r1 + r2;
        int64_t mid = r0 + (off[c + 1] - r0) / 2;   // child c1 = [r0, mid)
        for (int e = threadIdx.x; e < m * s; e += NT) {
            int i = e / s, col = e % s;
            int64_t a, b;
            int ii;
            if (i < r1) { a = r0; b = mid; ii = i; }
            else { a = mid; b = off[c + 1]; ii = i - r1; }
            double acc = 0.0;
            for (int64_t p = a; p < b; ++p) acc += Echild[p * rbc + ii] * Ylev[p * s + col];
            Yh[(size_t)i * s + col] = acc;
        }
    }
    __syncthreads();
    int k = cta_pivqr<NT>(Yh, s, m, s, tol, cap, V, dq, red, redi);
    // Frobenius norm of what the truncation left out: after k reflections the
    // not-yet-pivoted remainder of the sketch sits in Yh[k:m, k:s]; it is
    // <= tol unless the rank cap stopped the QR first
    double rem = 0.0;
    for (int e = threadIdx.x; e < (m - k) * (s - k); e += NT) {
        const double y = Yh[(size_t)(k + e / (s - k)) * s + k + e % (s - k)];
        rem += y * y;
    }
    rem = block_sum<NT>(rem, red);
    double* Q = Qout + (size_t)c * dq * dq;
    cta_form_q<NT>(Q, dq, m, V, dq, k);
    if (threadIdx.x == 0) {
        rank_out[c] = k;
        resid_out[c] = sqrt(rem);
    }
}

// E at this level (n x rbl, tree order rows): leaf E = Q[:, :r]; upper
// E_P = [E_c1 T[:r1, :rP]; E_c2 T[r1:, :rP]]
__global__ void k_expand(const int64_t* off, int leaf_level, const double* Q, int dq,
                         const int* rb, int rbl, const double* Echild, int rbc,
                         const int* rb_child, double* E) {
    int c = blockIdx.x;
    int64_t r0 = off[c], r1e = off[c + 1];
    int r = rb[c];
    const double* Qc = Q + (size_t)c * dq * dq;
    int64_t sz = r1e - r0;
    for (int64_t e = threadIdx.x; e < sz * rbl; e += NT) {
        int64_t p = r0 + e / rbl;
        int j = (int)(e % rbl);
        double v = 0.0;
        if (j < r) {
            if (leaf_level) {
                v = Qc[(size_t)(p - r0) * dq + j];
            } else {
                int c1 = 2 * c;
                int rr1 = rb_child[c1];
                int64_t mid = r0 + sz / 2;
                if (p < mid) {
                    for (int t = 0; t < rr1; ++t) v += Echild[p * rbc + t] * Qc[(size_t)t * dq + j];
                } else {
                    int rr2 = rb_child[c1 + 1];
                    for (int t = 0; t < rr2; ++t)
                        v += Echild[p * rbc + t] * Qc[(size_t)(rr1 + t) * dq + j];
                }
            }
        }
        E[p * rbl + j] = v;
    }
}

// couplings C_cd = E_c^T A(c,d) E_d for far pairs c > d; grid (pair, row chunk)
__global__ void k_coupling(KernelSpec ks, const double* __restrict__ X, const int64_t* off,
                           const int* pc, const int* pd, const double* E, int rbl, const int* rb,
                           double* C, int chunk) {
    int pi = blockIdx.x;
    int c = pc[pi], d = pd[pi];
    int rc = rb[c], rd = rb[d];
    int64_t a0 = off[c] + (int64_t)blockIdx.y * chunk;
    int64_t a1 = min(off[c + 1], a0 + chunk);
    if (a0 >= a1) return;
    extern __shared__ double sh[];        // t: chunk x rd, then acc rc x rd
    double* t = sh;
    double* acc = sh + (size_t)chunk * rbl;
    int rows = (int)(a1 - a0);
    for (int e = threadIdx.x; e < rows * rd; e += NT) {
        int i = e / rd, j = e % rd;
        const double* xi = X + 3 * (a0 + i);
        double v = 0.0;
        for (int64_t q = off[d]; q < off[d + 1]; ++q) v += kernel_entry(ks, xi, X + 3 * q) * E[q * rbl + j];
        t[(size_t)i * rbl + j] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rc * rd; e += NT) {
        int i = e / rd, j = e % rd;
        double v = 0.0;
        for (int p = 0; p < rows; ++p) v += E[(a0 + p) * rbl + i] * t[(size_t)p * rbl + j];
        acc[e] = v;
    }
    __syncthreads();
    double* Co = C + (size_t)pi * rbl * rbl;
    for (int e = threadIdx.x; e < rc * rd; e += NT) {
        int i = e / rd, j = e % rd;
        atomicAdd(&Co[(size_t)i * rbl + j], acc[e]);
    }
}

// leaf near blocks B = Q_c^T A(c,d) Q_d (slot-indexed, near slots only)
__global__ void k_near(KernelSpec ks, const double* __restrict__ X, const int64_t* off,
                       const int* slot_a, const int* slot_b, const int* slot_kind, const double* Q,
                       int dq, int dm, double* tmp, double* B) {
    int sl = blockIdx.x;
    if (slot_kind[sl] != 0) return;
    int c = slot_a[sl], d = slot_b[sl];
    int mc = (int)(off[c + 1] - off[c]), md = (int)(off[d + 1] - off[d]);
    double* A = tmp + (size_t)sl * 2 * dm * dm;
    double* T = A + (size_t)dm * dm;
    for (int e = threadIdx.x; e < mc * md; e += NT) {
        int i = e / md, j = e % md;
        A[(size_t)i * dm + j] = kernel_entry(ks, X + 3 * (off[c] + i), X + 3 * (off[d] + j));
    }
    __syncthreads();
    const double* Qd = Q + (size_t)d * dq * dq;
    const double* Qc = Q + (size_t)c * dq * dq;
    for (int e = threadIdx.x; e < mc * md; e += NT) {   // T = A Q_d
        int i = e / md, j = e % md;
        double v = 0.0;
        for (int p = 0; p < md; ++p) v += A[(size_t)i * dm + p] * Qd[(size_t)p * dq + j];
        T[(size_t)i * dm + j] = v;
    }
    __syncthreads();
    double* Bo = B + (size_t)sl * dm * dm;
    for (int e = threadIdx.x; e < dm * dm; e += NT) {   // B = Q_c^T T
        int i = e / dm, j = e % dm;
        double v = 0.0;
        if (i < mc && j < md)
            for (int p = 0; p < mc; ++p) v += Qc[(size_t)p * dq + i] * T[(size_t)p * dm + j];
        Bo[e] = v;
    }
}

// ---------------------------------------------------------------- driver --
int build_device(h2_matrix* h) {
    const Plan& P = h->plan;
    int L = P.L;
    int64_t n = P.n;
    cudaStream_t st = h->stream;
    KernelSpec ks{h->kernel.kind, h->kernel.p[0], h->kernel.p[1], h->kernel.p[2], h->kernel.p[3]};
    // points in tree order, padded to 3 coordinates
    std::vector<double> X(3 * n, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < P.d; ++k) X[3 * i + k] = h->plan_points[P.perm[i] * P.d + k];
    int rc = upload(&h->d_points, X);
    if (rc) return rc;
    // ||A||_inf and the Gershgorin interval
    double *d_rowabs, *d_diag, *d_g;
    if ((rc = dalloc(&d_rowabs, n)) || (rc = dalloc(&d_diag, n)) || (rc = dalloc(&d_g, 3))) return rc;
    k_rowsum<<<(unsigned)n, NT, 0, st>>>(ks, h->d_points, n, d_rowabs, d_diag);
    k_gershgorin<<<1, NT, 0, st>>>(d_rowabs, d_diag, n, d_g);
    double g[3];
    CK(cudaMemcpyAsync(g, d_g, sizeof(g), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    cudaFree(d_rowabs); cudaFree(d_diag); cudaFree(d_g);
    h->norm_inf = g[0]; h->glo = g[1]; h->ghi = g[2];
    h->tol = h->opt.eps_h2 * h->norm_inf;

    const int s = h->opt.sketch_cols > 0 ? h->opt.sketch_cols : h->rank + 16;
    const int cap = h->rank;
    const auto& leafp = P.lev[L];
    int nleaf = leafp.nc;
    int mmax = 0;
    for (int c = 0; c < nleaf; ++c) mmax = std::max<int>(mmax, (int)(leafp.off[c + 1] - leafp.off[c]));
    h->mmax = mmax;
    // sketch matrix
    double* d_Om;
    if ((rc = dalloc(&d_Om, (size_t)n * s))) return rc;
    k_omega<<<(unsigned)((n * s + NT - 1) / NT), NT, 0, st>>>(d_Om, n, s, h->opt.seed, std::sqrt(3.0 / s));
    // deepest near level h(tau, sigma) for every leaf pair
    std::vector<int> wl_tau, wl_h, wl_ptr{0}, wl_sigma;
    {
        std::vector<std::vector<int>> bylev(L > 0 ? L : 1);
        for (int tau = 0; tau < nleaf; ++tau) {
            for (auto& v : bylev) v.clear();
            for (int sg = 0; sg < nleaf; ++sg) {
                int hh = -1;
                for (int l = L; l >= 0; --l) {
                    const auto& lv = P.lev[l];
                    if (lv.is_near(tau >> (L - l), sg >> (L - l))) { hh = l; break; }
                }
                if (hh < L) bylev[hh].push_back(sg);
            }
            for (int hh = 0; hh < L; ++hh) {
                if (bylev[hh].empty()) continue;
                wl_tau.push_back(tau);
                wl_h.push_back(hh);
                wl_sigma.insert(wl_sigma.end(), bylev[hh].begin(), bylev[hh].end());
                wl_ptr.push_back((int)wl_sigma.size());
            }
        }
    }
    std::vector<int64_t> leaf_off(leafp.off.begin(), leafp.off.end());
    int64_t* d_leaf_off;
    int *d_wl_tau, *d_wl_h, *d_wl_ptr, *d_wl_sigma;
    double* d_Z;
    if ((rc = upload(&d_leaf_off, leaf_off)) || (rc = upload(&d_wl_tau, wl_tau)) ||
        (rc = upload(&d_wl_h, wl_h)) || (rc = upload(&d_wl_ptr, wl_ptr)) ||
        (rc = upload(&d_wl_sigma, wl_sigma)))
        return rc;
    size_t zsz = (size_t)nleaf * std::max(L, 1) * mmax * s;
    if ((rc = dalloc(&d_Z, zsz))) return rc;
    CK(cudaMemsetAsync(d_Z, 0, zsz * sizeof(double), st));
    if (!wl_tau.empty())
        k_sketch<<<(unsigned)wl_tau.size(), NT, 0, st>>>(ks, h->d_points, d_Om, s, d_leaf_off, d_wl_tau,
                                                        d_wl_h, d_wl_ptr, d_wl_sigma, std::max(L, 1),
                                                        mmax, d_Z);
    double* d_Y;
    if ((rc = dalloc(&d_Y, (size_t)n * s))) return rc;

    // bases, bottom-up
    h->lev.assign(L + 1, LevelDev());
    std::vector<double*> d_E(L + 1, nullptr);
    h->max_rank = 0;
    for (int l = L; l >= 0; --l) {
        LevelDev& D = h->lev[l];
        const LevelPlan& lp = P.lev[l];
        D.nc = lp.nc;
        int leaf_level = (l == L);
        int rbc = leaf_level ? 0 : h->lev[l + 1].estride;
        D.dq = leaf_level ? mmax : std::max(1, 2 * h->lev[l + 1].rbmax);
        std::vector<int64_t> off(lp.off.begin(), lp.off.end());
        int64_t* d_off;
        if ((rc = upload(&d_off, off))) return rc;
        k_sum_levels<<<nleaf, NT, 0, st>>>(d_Z, d_leaf_off, std::max(L, 1), mmax, s, l, d_Y);
        double* d_scr;
        if ((rc = dalloc(&d_scr, (size_t)D.nc * ((size_t)D.dq * s + (size_t)D.dq * D.dq)))) return rc;
        if ((rc = dalloc(&D.d_Q, (size_t)D.nc * D.dq * D.dq))) return rc;
        if ((rc = dalloc(&D.d_rb, D.nc))) return rc;
        double* d_res;
        if ((rc = dalloc(&d_res, D.nc))) return rc;
        k_basis<<<D.nc, NT, 0, st>>>(d_Y, s, d_off, leaf_level,
                                                       leaf_level ? nullptr : d_E[l + 1], rbc,
                                                       leaf_level ? nullptr : h->lev[l + 1].d_rb, D.dq,
                                                       h->tol, cap, d_scr, D.d_Q, D.d_rb, d_res);
        D.rb.resize(D.nc);
        D.resid.resize(D.nc);
        CK(cudaMemcpyAsync(D.rb.data(), D.d_rb, D.nc * sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(D.resid.data(), d_res, D.nc * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        cudaFree(d_res);
        D.rbmax = 0;
        for (int c = 0; c < D.nc; ++c) D.rbmax = std::max(D.rbmax, D.rb[c]);
        h->max_rank = std::max(h->max_rank, D.rbmax);
        int rbl = std::max(D.rbmax, 1);
        D.estride = rbl;
        if ((rc = dalloc(&d_E[l], (size_t)n * rbl))) return rc;
        k_expand<<<D.nc, NT, 0, st>>>(d_off, leaf_level, D.d_Q, D.dq, D.d_rb, rbl,
                                      leaf_level ? nullptr : d_E[l + 1], rbc,
                                      leaf_level ? nullptr : h->lev[l + 1].d_rb, d_E[l]);
        cudaFree(d_scr);
        // couplings of far pairs (c > d)
        D.far_of.assign((size_t)D.nc * D.nc, -1);
        std::vector<int> pc, pd;
        for (int c = 0; c < D.nc; ++c)
            for (int e = 0; e < c; ++e)
                if (lp.is_far(c, e)) {
                    D.far_of[(size_t)c * D.nc + e] = (int)pc.size();
                    pc.push_back(c);
                    pd.push_back(e);
                }
        D.nfar = (int)pc.size();
        if ((rc = dalloc(&D.d_C, (size_t)std::max(D.nfar, 1) * rbl * rbl))) return rc;
        CK(cudaMemsetAsync(D.d_C, 0, (size_t)std::max(D.nfar, 1) * rbl * rbl * sizeof(double), st));
        if (D.nfar > 0 && D.rbmax > 0) {
            int64_t maxsz = 0;
            for (int c = 0; c < D.nc; ++c) maxsz = std::max<int64_t>(maxsz, lp.off[c + 1] - lp.off[c]);
            int chunk = 64;
            int *d_pc, *d_pd;
            if ((rc = upload(&d_pc, pc)) || (rc = upload(&d_pd, pd))) return rc;
            dim3 grid(D.nfar, (unsigned)((maxsz + chunk - 1) / chunk));
            size_t shm = ((size_t)chunk * rbl + (size_t)rbl * rbl) * sizeof(double);
            if (shm > 48 * 1024)
                CK(cudaFuncSetAttribute(k_coupling, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
            k_coupling<<<grid, NT, shm, st>>>(ks, h->d_points, d_off, d_pc, d_pd, d_E[l], rbl, D.d_rb,
                                              D.d_C, chunk);
            CK(cudaStreamSynchronize(st));
            cudaFree(d_pc); cudaFree(d_pd);
        }
        D.d_off = d_off;
        {
            int* d_col;
            if ((rc = upload(&d_col, lp.color))) return rc;
            D.d_color = d_col;
        }
    }
    // slots (near and fill pairs, c >= d) and leaf near blocks
    for (int l = 0; l <= L; ++l) {
        LevelDev& D = h->lev[l];
        const LevelPlan& lp = P.lev[l];
        D.slot_of.assign((size_t)D.nc * D.nc, -1);
        std::vector<int> kind, farid;
        for (int c = 0; c < D.nc; ++c)
            for (int e = 0; e <= c; ++e)
                if (lp.is_near(c, e) || lp.is_fill(c, e)) {
                    D.slot_of[(size_t)c * D.nc + e] = (int)D.slot_a.size();
                    D.slot_a.push_back(c);
                    D.slot_b.push_back(e);
                    kind.push_back(lp.is_near(c, e) ? 0 : 1);
                    farid.push_back(lp.is_near(c, e) ? -1 : D.far_of[(size_t)c * D.nc + e]);
                }
        D.nslots = (int)D.slot_a.size();
        if ((rc = upload(&D.d_slot_a, D.slot_a)) || (rc = upload(&D.d_slot_b, D.slot_b)) ||
            (rc = upload(&D.d_slot_kind, kind)) || (rc = upload(&D.d_slot_far, farid)))
            return rc;
    }
    {
        LevelDev& D = h->lev[L];
        int dm = mmax;
        double* d_tmp;
        if ((rc = dalloc(&d_tmp, (size_t)D.nslots * 2 * dm * dm))) return rc;
        if ((rc = dalloc(&D.d_near_static, (size_t)D.nslots * dm * dm))) return rc;
        k_near<<<D.nslots, NT, 0, st>>>(ks, h->d_points, D.d_off, D.d_slot_a, D.d_slot_b,
                                        D.d_slot_kind, D.d_Q, D.dq, dm, d_tmp, D.d_near_static);
        CK(cudaStreamSynchronize(st));
        cudaFree(d_tmp);
    }
    CK(cudaStreamSynchronize(st));
    for (int l = 0; l <= L; ++l) cudaFree(d_E[l]);
    cudaFree(d_Om); cudaFree(d_Z); cudaFree(d_Y);
    cudaFree(d_leaf_off); cudaFree(d_wl_tau); cudaFree(d_wl_h); cudaFree(d_wl_ptr); cudaFree(d_wl_sigma);
    CK(cudaGetLastError());
    return H2_OK;
}

}  // namespace h2
