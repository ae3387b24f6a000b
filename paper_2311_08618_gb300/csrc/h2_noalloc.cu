// h2_dense_inertia_noalloc: the Bunch-Kaufman inertia of small dense shifted
// matrices with all working memory in a static device array, for callers that
// cannot allocate (see include/h2eig.h).  The library allocates nothing here.
#include <cfloat>
#include <mutex>

#include "h2_device.cuh"
#include "h2_internal.h"

using namespace h2dev;

namespace {

// Working copies of A - sigma I, one n x n slice per shift.  Shared by every
// call on a device; see the header for the race and size rules.
static __device__ __align__(256) double g_noalloc_scratch[H2_NOALLOC_MAX_DOUBLES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

constexpr int NT = 256;

// one CTA per shift: S = A - sigma I in the scratch slice, BK LDL^T in place
__global__ void __launch_bounds__(NT) k_dense_inertia(const double* __restrict__ A, int n, int lda,
                                                     const double* __restrict__ shifts, int64_t* counts,
                                                     double* minpiv, double* scratch) {
    extern __shared__ double sh_dbl[];
    double* bkbuf = sh_dbl;                       // 4n doubles
    int* perm = (int*)(sh_dbl + 4 * n);
    int* piv = perm + n;
    __shared__ double red[32];
    __shared__ int redi[32];
    __shared__ int s_neg, s_bad;
    __shared__ double s_mp;
    const int s = blockIdx.x;
    double* S = scratch + (size_t)s * n * n;
    const double sg = shifts[s];
    // ||A||_inf, for the exactly-zero pivot rule of the factorization: one
    // warp per row, its lanes striding along the row (coalesced reads)
    double rmax = 0.0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < n; i += NT / 32) {
        double r = 0.0;
        for (int j = lane; j < n; j += 32) r += fabs(A[(size_t)i * lda + j]);
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        rmax = fmax(rmax, r);
    }
    double dummy;
    int idx = block_argmax<NT>(rmax, threadIdx.x, red, redi, &dummy);
    (void)idx;
    const double norm = dummy;
    for (int e = threadIdx.x; e < n * n; e += NT) {
        int i = e / n, j = e % n;
        double v = A[(size_t)i * lda + j];
        if (i == j) v -= sg;
        S[e] = v;
    }
    if (threadIdx.x == 0) { s_neg = 0; s_bad = 0; s_mp = 1.0 / 0.0; }
    __syncthreads();
    cta_bk_ldl<NT>(S, n, n, perm, piv, red, redi, &s_neg, &s_mp, &s_bad, DBL_EPSILON * norm, bkbuf);
    if (threadIdx.x == 0) {
        counts[s] = s_neg;
        if (minpiv) minpiv[s] = s_bad ? __longlong_as_double(0x7ff8000000000000ll) : s_mp;
    }
}

// Set-up, once per device with that device current: the array's address.
int scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        h2::set_error(std::string("h2_dense_inertia_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return H2_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        h2::set_error("h2_dense_inertia_noalloc: device index out of range");
        return H2_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            h2::set_error(std::string("h2_dense_inertia_noalloc: cudaGetSymbolAddress: ") +
                          cudaGetErrorString(e));
            return H2_ERR_CUDA;
        }
        g_scratch_addr[dev] = (double*)p;
    }
    *out = g_scratch_addr[dev];
    return H2_OK;
}

}  // namespace

extern "C" int h2_dense_inertia_noalloc(const double* d_A, int n, int lda, const double* d_shifts, int ns,
                                        int64_t* d_counts, double* d_min_abs_pivot, void* stream) {
    if (!d_A || !d_shifts || !d_counts) {
        h2::set_error("h2_dense_inertia_noalloc: null pointer");
        return H2_ERR_INVALID_ARG;
    }
    if (n < 1 || n > 1024 || ns < 1 || ns > 1024 || lda < n) {
        h2::set_error("h2_dense_inertia_noalloc: need 1 <= n <= 1024, 1 <= ns <= 1024, lda >= n");
        return H2_ERR_INVALID_ARG;
    }
    if ((long long)ns * n * n > (long long)H2_NOALLOC_MAX_DOUBLES) {
        h2::set_error("h2_dense_inertia_noalloc: ns * n * n exceeds the static scratch of " +
                      std::to_string(H2_NOALLOC_MAX_DOUBLES) + " doubles");
        return H2_ERR_INVALID_ARG;
    }
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    k_dense_inertia<<<ns, NT, 4 * n * sizeof(double) + 2 * n * sizeof(int), (cudaStream_t)stream>>>(
        d_A, n, lda, d_shifts, d_counts,
                                                                          d_min_abs_pivot, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        h2::set_error(std::string("h2_dense_inertia_noalloc: launch: ") + cudaGetErrorString(e));
        return H2_ERR_CUDA;
    }
    return H2_OK;
}
