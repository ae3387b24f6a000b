// The resident H^2 representation as data and as an operator: h2_export copies
// one level's bases, couplings and near blocks to the host, and
// h2_compression_error measures ||A - A~||_2 and ||A||_2 on the device by
// power iteration, with A~ x formed by the nested H^2 matrix-vector product
// of Sec. 3.1 (upward pass through the transfer matrices, skeleton couplings,
// downward pass) plus the dense near blocks, and A x by evaluating the kernel
// entries on the fly (Sec. 3.1: ||U^S U^S^T A_{l;c,+} - A_{l;c,+}|| <= eps_H2
// is the quantity the construction truncates; Sec. 5 compares A~ with A).
#include <algorithm>
#include <cmath>
#include <vector>

#include "h2_device.cuh"
#include "h2_internal.h"

using namespace h2dev;

namespace h2 {

#define CKM(x)                                                                      \
    do {                                                                            \
        cudaError_t e_ = (x);                                                       \
        if (e_ != cudaSuccess) {                                                    \
            set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x); \
            return e_ == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA;      \
        }                                                                           \
    } while (0)

// ------------------------------------------------------------------ export --
int run_export(h2_matrix* h, h2_export_buf* b) {
    const int L = h->plan.L;
    if (b->level < 0 || b->level > L) {
        set_error("h2_export: level outside 0..L");
        return H2_ERR_INVALID_ARG;
    }
    const int l = b->level;
    const LevelDev& D = h->lev[l];
    const LevelPlan& lp = h->plan.lev[l];
    const int nc = D.nc;
    const int es = D.estride;
    std::vector<int> fc, fd, nc_, nd_;
    std::vector<int> fid, nid;
    for (int c = 0; c < nc; ++c)
        for (int d = 0; d < c; ++d)
            if (D.far_of[(size_t)c * nc + d] >= 0) {
                fc.push_back(c);
                fd.push_back(d);
                fid.push_back(D.far_of[(size_t)c * nc + d]);
            }
    if (l == L)
        for (int s = 0; s < D.nslots; ++s)
            if (lp.is_near(D.slot_a[s], D.slot_b[s])) {
                nc_.push_back(D.slot_a[s]);
                nd_.push_back(D.slot_b[s]);
                nid.push_back(s);
            }
    b->nc = nc;
    b->dq = D.dq;
    b->nfar = (int)fc.size();
    b->rbmax = es;
    b->nnear = (int)nc_.size();
    b->dm = l == L ? h->mmax : 0;
    if (b->offsets)
        for (int c = 0; c <= nc; ++c) b->offsets[c] = lp.off[c];
    if (b->ranks)
        for (int c = 0; c < nc; ++c) b->ranks[c] = D.rb[c];
    if (b->residuals)
        for (int c = 0; c < nc; ++c) b->residuals[c] = D.resid.empty() ? 0.0 : D.resid[c];
    if (b->colours)
        for (int c = 0; c < nc; ++c) b->colours[c] = lp.color[c];
    if (b->Q) CKM(cudaMemcpy(b->Q, D.d_Q, (size_t)nc * D.dq * D.dq * sizeof(double), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < fc.size(); ++i) {
        if (b->far_pairs) {
            b->far_pairs[2 * i] = fc[i];
            b->far_pairs[2 * i + 1] = fd[i];
        }
        if (b->C)
            CKM(cudaMemcpy(b->C + i * (size_t)es * es, D.d_C + (size_t)fid[i] * es * es,
                           (size_t)es * es * sizeof(double), cudaMemcpyDeviceToHost));
    }
    const size_t dm = (size_t)h->mmax;
    for (size_t i = 0; i < nc_.size(); ++i) {
        if (b->near_pairs) {
            b->near_pairs[2 * i] = nc_[i];
            b->near_pairs[2 * i + 1] = nd_[i];
        }
        if (b->B)
            CKM(cudaMemcpy(b->B + i * dm * dm, D.d_near_static + (size_t)nid[i] * dm * dm, dm * dm * sizeof(double),
                           cudaMemcpyDeviceToHost));
    }
    return H2_OK;
}

// --------------------------------------------------------- H^2 mat-vec ------
constexpr int MT = 128;

// xh[c][j] = sum_i Q_c[i][j] x[off_c + i], j < r_c: the skeleton coordinates
// of the leaf vector pieces (U^S^T x)
__global__ void k_up_leaf(const double* Q, int dq, const int* rb, const int64_t* off, const double* x,
                          double* xh, int es) {
    const int c = blockIdx.x;
    const int64_t r0 = off[c];
    const int m = (int)(off[c + 1] - r0), r = rb[c];
    for (int j = threadIdx.x; j < r; j += MT) {
        double a = 0.0;
        for (int i = 0; i < m; ++i) a += Q[((size_t)c * dq + i) * dq + j] * x[r0 + i];
        xh[(size_t)c * es + j] = a;
    }
}

// xh_P = T_P[:, :r_P]^T [xh_c1; xh_c2]: the nested upward step (transfer matrices)
__global__ void k_up(const double* T, int dq, const int* rbP, const double* xhc, int esc, const int* rbc,
                     double* xhP, int esP) {
    const int P = blockIdx.x, c1 = 2 * P, c2 = 2 * P + 1;
    const int r1 = rbc[c1], r2 = rbc[c2], rp = rbP[P];
    for (int j = threadIdx.x; j < rp; j += MT) {
        double a = 0.0;
        for (int i = 0; i < r1; ++i) a += T[((size_t)P * dq + i) * dq + j] * xhc[(size_t)c1 * esc + i];
        for (int i = 0; i < r2; ++i) a += T[((size_t)P * dq + r1 + i) * dq + j] * xhc[(size_t)c2 * esc + i];
        xhP[(size_t)P * esP + j] = a;
    }
}

// yh[c] = sum over far partners d of S_cd^SS xh[d] (couplings stored for c > d)
__global__ void k_far(const double* C, int es, const int* rb, const int* ptr, const int* other, const int* id,
                      const double* xh, double* yh) {
    const int c = blockIdx.x, rc = rb[c];
    for (int i = threadIdx.x; i < rc; i += MT) {
        double a = 0.0;
        for (int q = ptr[c]; q < ptr[c + 1]; ++q) {
            const int d = other[q], rd = rb[d];
            const double* Cq = C + (size_t)id[q] * es * es;
            if (c > d)
                for (int j = 0; j < rd; ++j) a += Cq[(size_t)i * es + j] * xh[(size_t)d * es + j];
            else
                for (int j = 0; j < rd; ++j) a += Cq[(size_t)j * es + i] * xh[(size_t)d * es + j];
        }
        yh[(size_t)c * es + i] = a;
    }
}

// yh_c += T_P[rows of c, :r_P] yh_P for both children: the downward step
__global__ void k_down(const double* T, int dq, const int* rbP, const double* yhP, int esP, const int* rbc,
                       double* yhc, int esc) {
    const int P = blockIdx.x, c1 = 2 * P;
    const int r1 = rbc[c1], r2 = rbc[c1 + 1], rp = rbP[P];
    for (int i = threadIdx.x; i < r1 + r2; i += MT) {
        double a = 0.0;
        for (int j = 0; j < rp; ++j) a += T[((size_t)P * dq + i) * dq + j] * yhP[(size_t)P * esP + j];
        const int c = i < r1 ? c1 : c1 + 1, ii = i < r1 ? i : i - r1;
        yhc[(size_t)c * esc + ii] += a;
    }
}

// y[off_c + i] = sum_j Q_c[i][j] yh_c[j] (j < r_c), then + the near-field part
// Q_c sum_d B_cd (Q_d^T x_d) with B_cd = Q_c^T A_cd Q_d (stored for c >= d)
__global__ void k_leaf_out(const double* Q, int dq, const int* rb, const int64_t* off, const double* yh, int es,
                           const double* B, int dm, const int* nptr, const int* nother, const int* nslot,
                           const double* t, double* u, double* y) {
    const int c = blockIdx.x;
    const int64_t r0 = off[c];
    const int m = (int)(off[c + 1] - r0), r = rb[c];
    double* uc = u + (size_t)c * dm;
    for (int i = threadIdx.x; i < m; i += MT) {
        double a = 0.0;
        for (int q = nptr[c]; q < nptr[c + 1]; ++q) {
            const int d = nother[q];
            const int md = (int)(off[d + 1] - off[d]);
            const double* Bq = B + (size_t)nslot[q] * dm * dm;
            const double* td = t + (size_t)d * dm;
            if (c >= d)
                for (int j = 0; j < md; ++j) a += Bq[(size_t)i * dm + j] * td[j];
            else
                for (int j = 0; j < md; ++j) a += Bq[(size_t)j * dm + i] * td[j];
        }
        uc[i] = a + (i < r ? yh[(size_t)c * es + i] : 0.0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += MT) {
        double a = 0.0;
        for (int j = 0; j < m; ++j) a += Q[((size_t)c * dq + i) * dq + j] * uc[j];
        y[r0 + i] = a;
    }
}

// t_d = Q_d^T x_d (all m_d coordinates) for every leaf
__global__ void k_leaf_in(const double* Q, int dq, const int64_t* off, const double* x, double* t, int dm) {
    const int d = blockIdx.x;
    const int64_t r0 = off[d];
    const int m = (int)(off[d + 1] - r0);
    for (int j = threadIdx.x; j < m; j += MT) {
        double a = 0.0;
        for (int i = 0; i < m; ++i) a += Q[((size_t)d * dq + i) * dq + j] * x[r0 + i];
        t[(size_t)d * dm + j] = a;
    }
}

// y = A x with the kernel entries evaluated on the fly (one CTA per row),
// or y = A x - y_in when sub = 1 (the residual (A - A~) x)
__global__ void k_dense_mv(KernelSpec ks, const double* X, int64_t n, const double* x, double* y, int sub) {
    __shared__ double red[32];
    const int64_t i = blockIdx.x;
    const double* xi = X + 3 * i;
    double a = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += 256) a += kernel_entry(ks, xi, X + 3 * j) * x[j];
    a = block_sum<256>(a, red);
    if (threadIdx.x == 0) y[i] = sub ? a - y[i] : a;
}

// out[0] = ||y||_2; x = y / ||y|| (x untouched when y = 0).  One CTA.
__global__ void k_normalize(const double* y, double* x, int64_t n, double* out) {
    __shared__ double red[32];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 256) a += y[i] * y[i];
    a = sqrt(block_sum<256>(a, red));
    if (threadIdx.x == 0) out[0] = a;
    if (a > 0.0)
        for (int64_t i = threadIdx.x; i < n; i += 256) x[i] = y[i] / a;
}

namespace {
struct Csr {
    std::vector<int> ptr, other, id;
};

template <typename T>
int dup(T** p, const std::vector<T>& v) {
    const size_t n = std::max<size_t>(v.size(), 1);
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return H2_ERR_OOM;
    }
    if (!v.empty()) CKM(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return H2_OK;
}

// Device buffers of one evaluation of A~ x, freed on destruction.
struct MatvecBufs {
    std::vector<void*> ptrs;
    ~MatvecBufs() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    int vec(T** p, const std::vector<T>& v) {
        int rc = dup(p, v);
        if (rc == H2_OK) ptrs.push_back(*p);
        return rc;
    }
    int zeros(double** p, size_t n) { return vec(p, std::vector<double>(std::max<size_t>(n, 1), 0.0)); }
};
}  // namespace

// ||A - A~||_2 and ||A||_2 by `iters` power-iteration steps each, from a
// seeded start vector (SplitMix64, state 0x9E37); everything in tree order.
int run_compression_error(h2_matrix* h, int iters, double* err2, double* norm2) {
    const Plan& P = h->plan;
    const int L = P.L;
    const int64_t n = h->n;
    cudaStream_t st = h->stream;
    KernelSpec ks{h->kernel.kind, h->kernel.p[0], h->kernel.p[1], h->kernel.p[2], h->kernel.p[3]};
    CKM(cudaStreamSynchronize(st));
    MatvecBufs bufs;
    int rc;
    // per level: skeleton vectors xh, yh ([nc][es]) and the far-pair lists
    std::vector<double*> xh(L + 1), yh(L + 1);
    std::vector<int*> fptr(L + 1), foth(L + 1), fid(L + 1);
    for (int l = 0; l <= L; ++l) {
        const LevelDev& D = h->lev[l];
        Csr f;
        f.ptr.push_back(0);
        for (int c = 0; c < D.nc; ++c) {
            for (int d = 0; d < D.nc; ++d) {
                const int id = c > d ? D.far_of[(size_t)c * D.nc + d] : (c < d ? D.far_of[(size_t)d * D.nc + c] : -1);
                if (id >= 0) {
                    f.other.push_back(d);
                    f.id.push_back(id);
                }
            }
            f.ptr.push_back((int)f.other.size());
        }
        if ((rc = bufs.zeros(&xh[l], (size_t)D.nc * D.estride)) || (rc = bufs.zeros(&yh[l], (size_t)D.nc * D.estride)) ||
            (rc = bufs.vec(&fptr[l], f.ptr)) || (rc = bufs.vec(&foth[l], f.other)) || (rc = bufs.vec(&fid[l], f.id)))
            return rc;
    }
    // leaf near lists
    const LevelDev& DL = h->lev[L];
    const LevelPlan& lpL = P.lev[L];
    Csr nr;
    nr.ptr.push_back(0);
    for (int c = 0; c < DL.nc; ++c) {
        for (int d = 0; d < DL.nc; ++d)
            if (lpL.is_near(c, d)) {
                nr.other.push_back(d);
                nr.id.push_back(DL.slot_of[(size_t)std::max(c, d) * DL.nc + std::min(c, d)]);
            }
        nr.ptr.push_back((int)nr.other.size());
    }
    int *nptr, *noth, *nslot;
    double *t, *u, *x, *y, *nrm;
    const int dm = h->mmax;
    if ((rc = bufs.vec(&nptr, nr.ptr)) || (rc = bufs.vec(&noth, nr.other)) || (rc = bufs.vec(&nslot, nr.id)) ||
        (rc = bufs.zeros(&t, (size_t)DL.nc * dm)) || (rc = bufs.zeros(&u, (size_t)DL.nc * dm)) ||
        (rc = bufs.zeros(&y, n)) || (rc = bufs.zeros(&nrm, 1)))
        return rc;
    std::vector<double> x0(n);
    uint64_t z = 0x9E37;
    for (int64_t i = 0; i < n; ++i) {         // SplitMix64 (Vigna): the start vector
        uint64_t q = (z += 0x9E3779B97F4A7C15ull);
        q = (q ^ (q >> 30)) * 0xBF58476D1CE4E5B9ull;
        q = (q ^ (q >> 27)) * 0x94D049BB133111EBull;
        q ^= q >> 31;
        x0[i] = (double)(q >> 11) * 0x1.0p-53 - 0.5;
    }
    if ((rc = bufs.vec(&x, x0))) return rc;
    const unsigned nb = (unsigned)n;
    // y = A~ x
    auto h2mv = [&]() {
        const LevelDev& Dl = h->lev[L];
        k_up_leaf<<<Dl.nc, MT, 0, st>>>(Dl.d_Q, Dl.dq, Dl.d_rb, Dl.d_off, x, xh[L], Dl.estride);
        for (int l = L - 1; l >= 0; --l) {
            const LevelDev& Dp = h->lev[l];
            const LevelDev& Dc = h->lev[l + 1];
            k_up<<<Dp.nc, MT, 0, st>>>(Dp.d_Q, Dp.dq, Dp.d_rb, xh[l + 1], Dc.estride, Dc.d_rb, xh[l], Dp.estride);
        }
        for (int l = 0; l <= L; ++l) {
            const LevelDev& D = h->lev[l];
            k_far<<<D.nc, MT, 0, st>>>(D.d_C, D.estride, D.d_rb, fptr[l], foth[l], fid[l], xh[l], yh[l]);
        }
        for (int l = 0; l < L; ++l) {
            const LevelDev& Dp = h->lev[l];
            const LevelDev& Dc = h->lev[l + 1];
            k_down<<<Dp.nc, MT, 0, st>>>(Dp.d_Q, Dp.dq, Dp.d_rb, yh[l], Dp.estride, Dc.d_rb, yh[l + 1], Dc.estride);
        }
        k_leaf_in<<<Dl.nc, MT, 0, st>>>(Dl.d_Q, Dl.dq, Dl.d_off, x, t, dm);
        k_leaf_out<<<Dl.nc, MT, 0, st>>>(Dl.d_Q, Dl.dq, Dl.d_rb, Dl.d_off, yh[L], Dl.estride, Dl.d_near_static, dm,
                                         nptr, noth, nslot, t, u, y);
    };
    double e_est = 0.0, a_est = 0.0;
    for (int it = 0; it < iters; ++it) {      // (A - A~) is symmetric: ||(A - A~) x|| -> ||A - A~||_2
        h2mv();
        k_dense_mv<<<nb, 256, 0, st>>>(ks, h->d_points, n, x, y, 1);
        k_normalize<<<1, 256, 0, st>>>(y, x, n, nrm);
    }
    CKM(cudaMemcpyAsync(&e_est, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
    CKM(cudaMemcpyAsync(x, x0.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    for (int it = 0; it < iters; ++it) {
        k_dense_mv<<<nb, 256, 0, st>>>(ks, h->d_points, n, x, y, 0);
        k_normalize<<<1, 256, 0, st>>>(y, x, n, nrm);
    }
    CKM(cudaMemcpyAsync(&a_est, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
    CKM(cudaStreamSynchronize(st));
    CKM(cudaGetLastError());
    *err2 = e_est;
    *norm2 = a_est;
    return H2_OK;
}

}  // namespace h2
