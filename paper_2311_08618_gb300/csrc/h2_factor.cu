// Per-shift generalized H^2-LDL^T factorization and inertia count on the device
// (Sec. 3.2-3.4 and Sec. 4), and the multi-interval bisection driver
// (Algorithm 1 with the inertia reuse of Sec. 4.2).
//
// One batch factorizes `lanes` shifted matrices A~ - sigma_b I at once.  Per
// level (leaves first) and per colour of the level's distance-2 colouring:
//   k_recomp : one CTA per (cluster p, lane): pivoted QR of the redundant rows
//              of p's fill-in blocks -> rotation V of p's redundant coordinates
//              (recompression, Sec. 3.4);
//   k_rotate : one CTA per (block of row p, lane): apply V to that block, drop
//              the truncated rows of fill-in blocks;
//   k_ldl    : one CTA per (cluster, lane): Bunch-Kaufman LDL^T of S_pp^RR and
//              its negative-pivot count (Eq. blr2-diag-ldl);
//   k_trsm   : one CTA per (coupled block a, lane): W_a = S_ap^{.R} P L^{-T},
//              Y_a = W_a D^{-1} (Eq. blr2-diag-elimination);
//   k_schur  : S_ab -= W_a Y_b^T on every pair of those blocks (Eq. blr2-diag-schur),
//              tiled 32 x 32 per CTA;
// then k_merge gathers the children's skeleton blocks into the parent level
// and applies the transfer bases (Sec. 3.3).  The whole sequence is captured
// once into a CUDA graph and replayed per batch.
#include <algorithm>
#include <functional>
#include <tuple>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

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

constexpr int NT = 256;
constexpr int TS = 32;   // Schur tile
constexpr int TSF = 64;  // Schur tile of the mixed (FP32) path

// Diagnostic heartbeat (enabled by H2_HEARTBEAT=1): per kernel kind, CTAs
// started, threads finished, and the block indices of the last CTA started,
// in zero-copy host memory so that the host can read them while the device
// is busy.  Null (no cost beyond one load) otherwise.
__device__ unsigned int* g_hb = nullptr;
struct HbScope {
    unsigned int* p;
    __device__ explicit HbScope(int kind) : p(g_hb ? g_hb + 4 * kind : nullptr) {
        if (p && threadIdx.x == 0) {
            atomicAdd_system(p, 1u);
            p[2] = blockIdx.x;
            p[3] = blockIdx.y;
        }
    }
    __device__ ~HbScope() {
        if (p) atomicAdd_system(p + 1, 1u);
    }
};

// scratch layout of one elimination (offsets in doubles)
struct ScratchLayout {
    size_t z, vr, vq, tmp, f, iperm, hdr, w, y;
    // FP64_TC only (dk > 0): BF16 digit planes [target][digit][row][dk] of W
    // and Y (k padded with zero digits to dk, a multiple of 32) and the
    // largest biased exponent of every row [target][row]
    size_t wd, yd, we, ye;
    size_t vd, ve;     // FP64_TC: digit planes of V^T [digit][row][dk] and row exponents
    int dk;
    size_t total;
};

static ScratchLayout scratch_layout(int D, int nfill_max, int ntarg_max, bool digits) {
    ScratchLayout s{};
    size_t zcols = (size_t)std::max(nfill_max, 1) * D;
    size_t o = 0;
    auto al = [&]() { o = (o + 3) & ~(size_t)3; };   // 32-byte aligned regions
    s.z = o; o += (size_t)D * zcols; al();
    s.vr = o; o += (size_t)D * D; al();
    s.vq = o; o += (size_t)D * D; al();
    s.tmp = o; o += (size_t)D * D; al();
    s.f = o; o += (size_t)D * D; al();
    s.iperm = o; o += (size_t)D; al();              // 2*D ints
    s.hdr = o; o += 8 + (size_t)(ntarg_max + 1) / 2 + 1; al();   // ints
    s.w = o; o += (size_t)ntarg_max * D * D; al();
    s.y = o; o += (size_t)ntarg_max * D * D; al();
    if (digits) {
        s.dk = (D + 31) / 32 * 32;
        const size_t plane = (size_t)ntarg_max * 8 * D * s.dk / 4;    // halves -> doubles
        s.wd = o; o += plane; al();
        s.yd = o; o += plane; al();
        s.we = o; o += ((size_t)ntarg_max * D + 1) / 2; al();
        s.ye = o; o += ((size_t)ntarg_max * D + 1) / 2; al();
        s.vd = o; o += (size_t)8 * D * s.dk / 4; al();
        s.ve = o; o += ((size_t)D + 1) / 2; al();
    }
    s.total = o;
    return s;
}

struct FactorArgs {
    double* slots;
    int D, lanes;
    int* dim;
    int* rk;
    const int* color;
    int cur_color;
    const int* cl;
    const int* targ;
    const int* targ_slot;
    const int* targ_trans;
    const int* ntarg;
    int ntarg_max;
    const int* rowblk;
    const int* rowblk_other;
    const int* rowblk_trans;
    const int* rowblk_fill;
    const int* nrow;
    int nrow_max;
    const int* fillq;
    const int* fillslot;
    const int* nfill;
    int nfill_max;
    double* scratch;
    ScratchLayout lay;
    double tol;
    double zero_pivot;
    int fill_cap;
    unsigned long long* neg;
    unsigned long long* minpiv;
    int* err;
    const int* active;
    double* stats;   // [2 * H2_NKINDS]: algorithmic flops, then bytes, per kernel kind
    int ncl;         // clusters of this colour
};

__device__ __forceinline__ double* slot_ptr(double* slots, int s, int lanes, int lane, int D) {
    return slots + ((size_t)s * lanes + lane) * (size_t)D * D;
}

// element (i, j) of block (x, y) stored as (x, y) (trans = 0) or as (y, x) (trans = 1)
__device__ __forceinline__ double& belem(double* B, int D, int trans, int i, int j) {
    return trans ? B[(size_t)j * D + i] : B[(size_t)i * D + j];
}

// Symmetric Schur updates.  The update of a diagonal block, S_aa -= W_a Y_a^T
// = W_a D^-1 W_a^T, is symmetric: only the tiles on and below the tile
// diagonal are computed, and each lower tile also writes its transpose into
// the skipped upper tile (the DFMA kernel computes only the lower triangle of
// a diagonal tile as well).  Live entries of an r x r block covered by the
// tiles on and below the tile diagonal (ts x ts):
__device__ __forceinline__ double lower_tile_entries(int r, int ts) {
    double s = 0.0;
    for (int i0 = 0; i0 < r; i0 += ts) s += (double)min(ts, r - i0) * min(r, i0 + ts);
    return s;
}

// S(j0 + c, i0 + r) -= T[r][c] for r < nr, c < nc: the mirror of lower tile
// (i0, j0) staged in shared memory (ld = leading dimension of T).  Threads
// run along r, so the writes are coalesced.  All threads of the CTA call it.
template <typename V>
__device__ __forceinline__ void schur_mirror(double* B, int D, int trans, int i0, int j0, int nr, int nc,
                                             const V* T, int ld, int rows_per_pass) {
    const int r = threadIdx.x % rows_per_pass;
    for (int c = threadIdx.x / rows_per_pass; c < nc; c += blockDim.x / rows_per_pass)
        if (r < nr) belem(B, D, trans, j0 + c, i0 + r) -= (double)T[(size_t)r * ld + c];
}

// rows of cluster x still in the trailing matrix: all of them until x is
// eliminated, its skeleton afterwards
__device__ __forceinline__ int live_rows(const FactorArgs& A, int x, int lane) {
    return A.color[x] < A.cur_color ? A.rk[x * A.lanes + lane] : A.dim[x * A.lanes + lane];
}

__device__ __forceinline__ void add_stats(double* stats, int kind, double fl, double by) {
    atomicAdd(&stats[kind], fl);
    atomicAdd(&stats[H2_NKINDS + kind], by);
}

// Self-check record (err[0..7]): err[0] |= 1 for NaN, |= 2 when a kernel
// meets a size outside its buffers (it then skips its work); the first such
// kernel writes its id, four values and its block indices into err[1..7].
__device__ __noinline__ void report_bad(int* err, int kernel, int a, int b, int c, int d) {
    atomicOr(&err[0], 2);
    if (atomicCAS(&err[1], 0, kernel) == 0) {
        err[2] = a;
        err[3] = b;
        err[4] = c;
        err[5] = d;
        err[6] = blockIdx.x;
        err[7] = blockIdx.y;
    }
}

// scratch header (ints): [0] rk after recompression, [1] R', [2] r0, [3] t,
// [4] recompression ran, [8 + ti] live rows of target ti
constexpr int HDR_ROWS = 8;

// Digits of the FP64_TC Schur products (see k_schur_oz).
constexpr int OZP = 8;
constexpr int OZK = 32;
constexpr int OZLD = OZK + 8;   // BF16 row stride: fragment loads hit 32 distinct banks

// biased exponent field of x (0 for zero and subnormals)
__device__ __forceinline__ int oz_expo(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7ff);
}

// the 8 BF16 digits of x for a row whose largest biased exponent is emax
__device__ __forceinline__ void oz_digits(double x, int emax, uint32_t (&d)[OZP]) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    unsigned long long F = 0;
    if (ex != 0) {
        const unsigned long long M = (b & 0xfffffffffffffull) | (1ull << 52);
        const int sh = ex - emax + 3;            // F = |x| 2^(56 - e) = M 2^sh < 2^56
        F = sh >= 0 ? (M << sh) : (sh > -64 ? (M >> -sh) : 0ull);
    }
    const uint32_t sg = (uint32_t)(b >> 48) & 0x8000u;
#pragma unroll
    for (int p = 0; p < OZP; ++p) {
        const uint32_t v = (uint32_t)(F >> (49 - 7 * p)) & 127u;
        const float f = __uint_as_float(0x4B000000u | v) - 8388608.0f;   // (float)v, exact
        d[p] = (__float_as_uint(f) >> 16) | (v ? sg : 0u);              // BF16 bits, exact
    }
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// an integer-valued float below 2^22 in magnitude, as int (exact)
__device__ __forceinline__ long long oz_int(float v) {
    return (long long)(__float_as_int(v + 12582912.0f) - 0x4B400000);
}

// One warp's 16 x 8 output piece (rows 16 mi.., columns 8 ni..) over kc <= OZK
// values of k: the 36 digit-pair products, folded exactly into hi / lo.
// Digit p of row r, column k of an operand sits at X + p * xp + r * xl + k.
__device__ __forceinline__ void oz_warp_chunk(const uint16_t* A, int ap, int al, const uint16_t* B, int bp, int bl,
                                              int mi, int ni, int kc, long long (&hi)[4], long long (&lo)[4]) {
    const int l = threadIdx.x % 32, gid = l / 4, tig = l % 4;
    float acc[OZP][4];
#pragma unroll
    for (int t = 0; t < OZP; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
    for (int s0 = 0; s0 < kc; s0 += 16) {
        uint32_t b[OZP][2];
#pragma unroll
        for (int q = 0; q < OZP; ++q) {
            const uint16_t* bq = B + q * bp + (8 * ni + gid) * bl + s0 + 2 * tig;
            b[q][0] = *reinterpret_cast<const uint32_t*>(bq);
            b[q][1] = *reinterpret_cast<const uint32_t*>(bq + 8);
        }
#pragma unroll
        for (int p = 0; p < OZP; ++p) {
            const uint16_t* ap0 = A + p * ap + (16 * mi + gid) * al + s0 + 2 * tig;
            uint32_t a[4];
            a[0] = *reinterpret_cast<const uint32_t*>(ap0);
            a[1] = *reinterpret_cast<const uint32_t*>(ap0 + 8 * al);
            a[2] = *reinterpret_cast<const uint32_t*>(ap0 + 8);
            a[3] = *reinterpret_cast<const uint32_t*>(ap0 + 8 * al + 8);
#pragma unroll
            for (int q = 0; q < OZP - p; ++q) mma_bf16(acc[p + q], a, b[q][0], b[q][1]);
        }
    }
    // level t = p + q + 2: hi gets t = 2..5, lo gets t = 6..9 (exact)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        long long h = oz_int(acc[0][c]);
        h = h * 128 + oz_int(acc[1][c]);
        h = h * 128 + oz_int(acc[2][c]);
        h = h * 128 + oz_int(acc[3][c]);
        long long g = oz_int(acc[4][c]);
        g = g * 128 + oz_int(acc[5][c]);
        g = g * 128 + oz_int(acc[6][c]);
        g = g * 128 + oz_int(acc[7][c]);
        hi[c] += h;
        lo[c] += g;
    }
}

// the FP64 value of a folded product: (hi 2^-35 + lo 2^-63) 2^(e_row + e_col),
// from the rows' largest biased exponents (one rounding)
__device__ __forceinline__ double oz_value(long long hi, long long lo, int erow, int ecol) {
    const int e = (erow - 1022) + (ecol - 1022) - 35;
    const double v = fma((double)lo, 0x1p-28, (double)hi);   // exact operands, one rounding
    const double sc = (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
    return v * sc;
}

// digit planes (row-scaled) of the R x R operand X^T for X = V: row i of
// X^T is column i of V (leading dimension ldv), written as [p][i][dk] with
// zero digits for k in [R, round32(R)); ve[i] = the row's largest exponent.
// All threads of the CTA call it.
__device__ void oz_planes_of_transpose(const double* V, int ldv, int R, int D, int dk, uint16_t* vd, int* ve) {
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    for (int i = w; i < R; i += blockDim.x / 32) {
        int e = 0;
        for (int k = l; k < R; k += 32) e = max(e, oz_expo(V[(size_t)k * ldv + i]));
        for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (l == 0) ve[i] = e;
    }
    __syncthreads();
    const int npair = (R + 31) / 32 * 16;
    for (int e = threadIdx.x; e < R * npair; e += blockDim.x) {
        const int i = e / npair, k = 2 * (e % npair);
        const double x0 = k < R ? V[(size_t)k * ldv + i] : 0.0;
        const double x1 = k + 1 < R ? V[(size_t)(k + 1) * ldv + i] : 0.0;
        uint32_t d0[OZP], d1[OZP];
        oz_digits(x0, ve[i], d0);
        oz_digits(x1, ve[i], d1);
#pragma unroll
        for (int p = 0; p < OZP; ++p)
            *reinterpret_cast<uint32_t*>(&vd[((size_t)p * D + i) * dk + k]) = d0[p] | (d1[p] << 16);
    }
    __syncthreads();
}

// Multi-matrix (grouped) launches.  A grouped launch runs one kernel over the
// work of several handles: item m (a handle's level and colour) owns the
// blockIdx.x range [off[m], off[m+1]) and its own argument struct; flag[m]
// carries the item's shared-memory switch where the kernel has one.  The
// kernel bodies take their block coordinates as arguments, so the single and
// the grouped launches execute the same code.
template <typename Args>
struct GroupArgs {
    const Args* args;
    const int* off;      // n + 1 prefix offsets of blockIdx.x
    const int* flag;     // per item (may be null)
    int n;
};

__device__ __forceinline__ int group_find(const int* off, int n, int bx) {
    int lo = 0, hi = n - 1;                      // largest m with off[m] <= bx
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= bx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---- (i) recompression basis of row p (Sec. 3.4): one CTA per (cluster, lane)
__device__ __forceinline__ void k_recomp_body(const FactorArgs& A, const int bx, const int by) {
    HbScope hb_(1);
    const int ci = bx, lane = by;
    if (lane >= *A.active) return;
    __shared__ double red[32];
    __shared__ int redi[32];
    __shared__ int s_bad;
    const int D = A.D, LN = A.lanes;
    const int p = A.cl[ci];
    const int m = A.dim[p * LN + lane], r0 = A.rk[p * LN + lane];
    double* scr = A.scratch + ((size_t)ci * LN + lane) * A.lay.total;
    double* Z = scr + A.lay.z;
    double* Vr = scr + A.lay.vr;
    double* Vq = scr + A.lay.vq;
    int* hdr = (int*)(scr + A.lay.hdr);
    const int R = m - r0;
    const int nf = A.nfill[ci];
    if (m < 0 || m > D || r0 < 0 || r0 > m || nf < 0 || nf > A.nfill_max) {
        if (threadIdx.x == 0) report_bad(A.err, 1, m, r0, nf, D);
        return;
    }
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    int t = 0;
    const int run = (nf > 0 && R > 0) ? 1 : 0;
    if (run) {
        int wz = 0, badq = -1;
        for (int f = 0; f < nf; ++f) {
            int lq = live_rows(A, A.fillq[ci * A.nfill_max + f], lane);
            if (lq < 0 || lq > D) badq = lq;
            wz += lq;
        }
        if (badq != -1) {
            if (threadIdx.x == 0) report_bad(A.err, 1, badq, wz, m, D);
            return;
        }
        int coff = 0;
        for (int f = 0; f < nf; ++f) {
            int q = A.fillq[ci * A.nfill_max + f];
            int lq = live_rows(A, q, lane);
            double* B = slot_ptr(A.slots, A.fillslot[ci * A.nfill_max + f], LN, lane, D);
            int tr = p > q ? 0 : 1;
            for (int e = threadIdx.x; e < R * lq; e += NT) {
                int i = e / lq, j = e % lq;
                Z[(size_t)i * wz + coff + j] = belem(B, D, tr, r0 + i, j);
            }
            coff += lq;
        }
        __syncthreads();
        int capt = max(0, min(A.fill_cap, m) - r0);
        t = cta_pivqr<NT>(Z, wz, R, wz, A.tol, capt, Vr, D, red, redi, &s_bad);
        if (t > 0) cta_form_q<NT>(Vq, D, R, Vr, D, t);
        if (t > 0 && A.lay.dk > 0)        // FP64_TC: digit planes of Vq^T for the rotation
            oz_planes_of_transpose(Vq, D, R, D, A.lay.dk, reinterpret_cast<uint16_t*>(scr + A.lay.vd),
                                   reinterpret_cast<int*>(scr + A.lay.ve));
        if (threadIdx.x == 0)
            add_stats(A.stats, H2_KIND_RECOMP, 4.0 * R * (double)wz * t + 4.0 * (double)R * R * t,
                      8.0 * 2.0 * R * (double)wz);
    }
    if (threadIdx.x == 0) {
        hdr[2] = r0;
        hdr[3] = t;
        hdr[4] = run;
        A.rk[p * LN + lane] = r0 + t;
        if (s_bad) atomicOr(A.err, 1);
    }
}
__global__ void __launch_bounds__(NT) k_recomp(FactorArgs A) { k_recomp_body(A, blockIdx.x, blockIdx.y); }
__global__ void __launch_bounds__(NT) k_recomp_g(GroupArgs<FactorArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_recomp_body(G.args[m], blockIdx.x - G.off[m], blockIdx.y);
}

// ---- (i') the same recompression for wide fill rows: one thread-block
// cluster of QG CTAs per (cluster, lane).  The columns of Z are split into QG
// contiguous ranges; per step the CTAs exchange their partial norm sums and
// pivot candidates through distributed shared memory, CTA 0 swaps the pivot
// column into place, and every CTA forms the same reflector from it and
// applies it to its own columns (fusing the norms of the next step, as
// cta_pivqr does).  The pivot rule (largest norm, then smallest index) does
// not depend on the split, so the reflectors equal those of cta_pivqr; only
// the addition order of the stopping sum differs.
namespace cg = cooperative_groups;
constexpr int QG = 8;
struct QPart {
    double total, best;
    int bi, pad;
};

__device__ int cluster_pivqr(cg::cluster_group& cl, int g, double* Y, int ldy, int m, int s, double tol, int cap,
                             double* V, int ldv, double* sv, double* red, int* redi, QPart* xs, int* bad) {
    const int cw = (s + QG - 1) / QG;
    const int jlo = g * cw, jhi = min(s, jlo + cw);
    const int kmax = min(min(m, s), cap);
    int par = 0, xp = 0, k = 0;
    double part = 0.0, best = -1.0;
    int bi = 0x7fffffff;
    for (int j = jlo + threadIdx.x; j < jhi; j += NT) {   // norms of step 0
        double a = 0.0;
        for (int i = 0; i < m; ++i) {
            double y = Y[(size_t)i * ldy + j];
            a += y * y;
        }
        part += a;
        if (a > best) { best = a; bi = j; }
    }
    for (; k < kmax; ++k) {
        const double ctot = block_sum1<NT>(part, red, par);
        par ^= 1;
        double cbv;
        const int cbi = block_argmax1<NT>(best, bi, red, redi, par, &cbv);
        par ^= 1;
        if (threadIdx.x == 0) {
            xs[xp].total = ctot;
            xs[xp].best = cbv;
            xs[xp].bi = cbi;
        }
        cl.sync();
        double total = 0.0, bv = -1.0;
        int jp = 0x7fffffff;
        for (int r = 0; r < QG; ++r) {       // the same order on every CTA
            const QPart* q = cl.map_shared_rank(&xs[xp], r);
            total += q->total;
            if (q->best > bv || (q->best == bv && q->bi < jp)) { bv = q->best; jp = q->bi; }
        }
        xp ^= 1;
        if (!(total == total)) {
            if (bad && threadIdx.x == 0 && g == 0) *bad = 1;
            break;
        }
        if (total <= tol * tol) break;
        if (jp < k || jp >= s) jp = k;
        if (g == 0 && jp != k)
            for (int i = threadIdx.x; i < m; i += NT) {
                double t = Y[(size_t)i * ldy + k];
                Y[(size_t)i * ldy + k] = Y[(size_t)i * ldy + jp];
                Y[(size_t)i * ldy + jp] = t;
            }
        cl.sync();
        // reflector from x = Y[k:, k], identical on every CTA; |x|^2 is the
        // winning column norm of the search
        const double nx2 = bv;
        const double nx = sqrt(nx2);
        const double x0 = Y[(size_t)k * ldy + k];
        const double alpha = x0 >= 0.0 ? -nx : nx;
        const double v0 = x0 - alpha;
        // |v|^2 = 2 |x|^2 + 2 |x0| |x|, as in cta_pivqr
        const double nv = sqrt(2.0 * nx2 + 2.0 * fabs(x0) * nx);
        const double inv_nv = nv > 0.0 ? 1.0 / nv : 0.0;
        for (int i = threadIdx.x; i < m; i += NT) {
            double x = 0.0;
            if (i >= k && nv > 0.0) x = ((i == k) ? v0 : Y[(size_t)i * ldy + k]) * inv_nv;
            sv[i] = x;
            if (g == 0) V[(size_t)i * ldv + k] = x;
        }
        __syncthreads();
        // own columns j > k: apply the reflector, norms of step k+1
        part = 0.0;
        best = -1.0;
        bi = 0x7fffffff;
        for (int j = max(jlo, k + 1) + threadIdx.x; j < jhi; j += NT) {
            double a = 0.0;
            if (nv > 0.0) {
                double w = 0.0;
                for (int i = k; i < m; ++i) w += sv[i] * Y[(size_t)i * ldy + j];
                w *= 2.0;
                Y[(size_t)k * ldy + j] -= w * sv[k];
                for (int i = k + 1; i < m; ++i) {
                    double y = Y[(size_t)i * ldy + j] - w * sv[i];
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
    cl.sync();     // V complete; no CTA leaves while others read its xs
    return k;
}

__device__ __forceinline__ void k_recomp_cluster_body(const FactorArgs& A, const int bx, const int by) {
    HbScope hb_(1);
    cg::cluster_group cl = cg::this_cluster();
    const int g = (int)cl.block_rank();
    const int ci = bx / QG, lane = by;
    // every early return below depends on (ci, lane) only: taken by the whole cluster
    if (lane >= *A.active) return;
    extern __shared__ double sv[];       // reflector, D doubles
    __shared__ double red[2 * NT / 32];
    __shared__ int redi[2 * NT / 32];
    __shared__ QPart xs[2];
    __shared__ int s_bad;
    const int D = A.D, LN = A.lanes;
    const int p = A.cl[ci];
    const int m = A.dim[p * LN + lane], r0 = A.rk[p * LN + lane];
    double* scr = A.scratch + ((size_t)ci * LN + lane) * A.lay.total;
    double* Z = scr + A.lay.z;
    double* Vr = scr + A.lay.vr;
    double* Vq = scr + A.lay.vq;
    int* hdr = (int*)(scr + A.lay.hdr);
    const int R = m - r0;
    const int nf = A.nfill[ci];
    if (m < 0 || m > D || r0 < 0 || r0 > m || nf < 0 || nf > A.nfill_max) {
        if (g == 0 && threadIdx.x == 0) report_bad(A.err, 1, m, r0, nf, D);
        return;
    }
    int wz = 0, badq = -1;
    for (int f = 0; f < nf; ++f) {
        int lq = live_rows(A, A.fillq[ci * A.nfill_max + f], lane);
        if (lq < 0 || lq > D) badq = lq;
        wz += lq;
    }
    if (badq != -1) {
        if (g == 0 && threadIdx.x == 0) report_bad(A.err, 1, badq, wz, m, D);
        return;
    }
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    int t = 0;
    const int run = (nf > 0 && R > 0) ? 1 : 0;
    if (run) {
        // Z = rows r0.. of every fill block of row p, assembled by the cluster
        int coff = 0;
        for (int f = 0; f < nf; ++f) {
            int q = A.fillq[ci * A.nfill_max + f];
            int lq = live_rows(A, q, lane);
            double* B = slot_ptr(A.slots, A.fillslot[ci * A.nfill_max + f], LN, lane, D);
            int tr = p > q ? 0 : 1;
            for (int e = g * NT + threadIdx.x; e < R * lq; e += QG * NT) {
                int i = e / lq, j = e % lq;
                Z[(size_t)i * wz + coff + j] = belem(B, D, tr, r0 + i, j);
            }
            coff += lq;
        }
        cl.sync();
        int capt = max(0, min(A.fill_cap, m) - r0);
        t = cluster_pivqr(cl, g, Z, wz, R, wz, A.tol, capt, Vr, D, sv, red, redi, xs, &s_bad);
        if (g == 0) {
            if (t > 0) cta_form_q<NT>(Vq, D, R, Vr, D, t);
            if (t > 0 && A.lay.dk > 0)
                oz_planes_of_transpose(Vq, D, R, D, A.lay.dk, reinterpret_cast<uint16_t*>(scr + A.lay.vd),
                                       reinterpret_cast<int*>(scr + A.lay.ve));
            if (threadIdx.x == 0)
                add_stats(A.stats, H2_KIND_RECOMP, 4.0 * R * (double)wz * t + 4.0 * (double)R * R * t,
                          8.0 * 2.0 * R * (double)wz);
        }
    }
    if (g == 0 && threadIdx.x == 0) {
        hdr[2] = r0;
        hdr[3] = t;
        hdr[4] = run;
        A.rk[p * LN + lane] = r0 + t;
        if (s_bad) atomicOr(A.err, 1);
    }
}
__global__ void __cluster_dims__(QG, 1, 1) __launch_bounds__(NT) k_recomp_cluster(FactorArgs A) {
    k_recomp_cluster_body(A, blockIdx.x, blockIdx.y);
}
// item offsets are multiples of QG, so a cluster never spans two items
__global__ void __cluster_dims__(QG, 1, 1) __launch_bounds__(NT) k_recomp_cluster_g(GroupArgs<FactorArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_recomp_cluster_body(G.args[m], blockIdx.x - G.off[m], blockIdx.y);
}

// ---- (ii) rotation of p's redundant coordinates in one block of row p and
// truncation of a fill-in block: one CTA per (row block, cluster, lane)
constexpr int RC = 32;   // columns (or rows) of the block rotated per pass
constexpr int RK = 32;   // rows of V staged in shared memory per step

// VEC consecutive T values from shared memory (VEC * sizeof(T)-byte aligned)
__device__ __forceinline__ void ldsv(const float* p, float (&v)[2]) {
    float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x; v[1] = q.y;
}
__device__ __forceinline__ void ldsv(const double* p, double (&v)[1]) { v[0] = *p; }

// out(i, c) = sum_k V[k][ib + i] * slab[k][c] for the column c = tx and the
// rows i = VEC*ty + 8*VEC*g + u (u < VEC, g < ng) of one pass over up to 8*NU
// rows starting at ib; V is the R x R rotation in global memory (leading
// dimension D), staged RK rows at a time in vs (leading dimension 8*NU) in the
// product type T.  VEC = 2 for float (pairs of rows per load), 1 for double;
// ng = the row groups this pass needs, so no padded rows are computed beyond
// the last group of 8*VEC rows.
template <typename T, int NU>
__device__ __forceinline__ void rot_product(const T* slab, T* vs, const double* V, int D, int R, int ib,
                                            T (&acc)[NU]) {
    constexpr int VEC = sizeof(T) == 4 ? 2 : 1;
    constexpr int LDV = 8 * NU;
    constexpr int G = NU / VEC;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    const int ng = min(G, (R - ib + 8 * VEC - 1) / (8 * VEC));
#pragma unroll
    for (int u = 0; u < NU; ++u) acc[u] = (T)0;
    for (int k0 = 0; k0 < R; k0 += RK) {
        const int kc = min(RK, R - k0);
        for (int e = threadIdx.x; e < RK * LDV; e += NT) {
            int k = e / LDV, i = e % LDV;
            vs[e] = (k < kc && ib + i < R) ? (T)V[(size_t)(k0 + k) * D + ib + i] : (T)0;
        }
        __syncthreads();
        for (int k = 0; k < kc; ++k) {
            const T y = slab[(k0 + k) * RC + tx];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (g < ng) {
                    T v[VEC];
                    ldsv(vs + k * LDV + 8 * VEC * g + VEC * ty, v);
#pragma unroll
                    for (int u = 0; u < VEC; ++u) acc[VEC * g + u] += v[u] * y;
                }
            }
        }
        __syncthreads();
    }
}

// row of pass-local output u of this thread (see rot_product)
template <typename T>
__device__ __forceinline__ int rot_row(int u) {
    constexpr int VEC = sizeof(T) == 4 ? 2 : 1;
    return VEC * (threadIdx.x / 32) + 8 * VEC * (u / VEC) + u % VEC;
}

// Rotates rows r0.. of block B (row side) or its columns r0.. (column side of
// the diagonal block) by V, in passes of RC columns (rows) staged in slab.
template <typename T, int NU>
__device__ void rotate_block(double* B, int D, int tr, int r0, int R, int dx, int m, const double* V, T* slab,
                             T* vs) {
    const int tx = threadIdx.x % 32;
    T acc[NU];
    // row side: rows r0.. of p, over the dx live columns of x
    for (int j0 = 0; j0 < dx; j0 += RC) {
        const int nj = min(RC, dx - j0);
        for (int e = threadIdx.x; e < R * RC; e += NT) {
            int k, j;
            if (tr) { j = e / R; k = e % R; } else { k = e / RC; j = e % RC; }
            slab[k * RC + j] = j < nj ? (T)belem(B, D, tr, r0 + k, j0 + j) : (T)0;
        }
        __syncthreads();
        for (int ib = 0; ib < R; ib += 8 * NU) {
            rot_product<T, NU>(slab, vs, V, D, R, ib, acc);
            if (tx < nj) {
#pragma unroll
                for (int u = 0; u < NU; ++u) {
                    int i = ib + rot_row<T>(u);
                    if (i < R) belem(B, D, tr, r0 + i, j0 + tx) = (double)acc[u];
                }
            }
        }
        __syncthreads();
    }
    if (m < 0) return;
    // column side (diagonal block only): columns r0.. for every row
    for (int i0 = 0; i0 < m; i0 += RC) {
        const int ni = min(RC, m - i0);
        for (int e = threadIdx.x; e < R * RC; e += NT) {
            int i = e / R, k = e % R;
            slab[k * RC + i] = i < ni ? (T)B[(size_t)(i0 + i) * D + r0 + k] : (T)0;
        }
        __syncthreads();
        for (int jb = 0; jb < R; jb += 8 * NU) {
            rot_product<T, NU>(slab, vs, V, D, R, jb, acc);
            if (tx < ni) {
#pragma unroll
                for (int u = 0; u < NU; ++u) {
                    int j = jb + rot_row<T>(u);
                    if (j < R) B[(size_t)(i0 + tx) * D + r0 + j] = (double)acc[u];
                }
            }
        }
        __syncthreads();
    }
}

// row groups of k_rotate (8 * NU rows per pass) for blocks of dimension D
__host__ __device__ constexpr int rotate_nu(int D) { return D <= 64 ? 8 : D <= 128 ? 16 : 32; }

// shared memory of k_rotate for blocks of dimension at most D
template <typename T>
__host__ __device__ constexpr size_t rotate_smem(int D) {
    return ((size_t)D * RC + (size_t)RK * 8 * rotate_nu(D)) * sizeof(T);
}

// NU = rotate_nu(D) of the level (R <= D; rows beyond 8 * NU take more passes)
template <typename T, int NU>
__device__ __forceinline__ void k_rotate_body(const FactorArgs& A, const int bx, const int by) {
    HbScope hb_(2);
    const int ci = bx / A.nrow_max, b = bx % A.nrow_max, lane = by;
    if (lane >= *A.active || b >= A.nrow[ci]) return;
    extern __shared__ __align__(16) unsigned char rot_smem[];
    const int D = A.D, LN = A.lanes;
    const int p = A.cl[ci];
    const double* scr = A.scratch + ((size_t)ci * LN + lane) * A.lay.total;
    const int* hdr = (const int*)(scr + A.lay.hdr);
    if (!hdr[4]) return;
    const int r0 = hdr[2], t = hdr[3];
    const int m = A.dim[p * LN + lane];
    const int R = m - r0;
    const double* Vq = scr + A.lay.vq;
    const int x = A.rowblk_other[ci * A.nrow_max + b];
    const int tr = A.rowblk_trans[ci * A.nrow_max + b];
    double* B = slot_ptr(A.slots, A.rowblk[ci * A.nrow_max + b], LN, lane, D);
    {
        const int dxl = live_rows(A, x, lane), dqa = A.dim[x * LN + lane];
        if (m < 0 || m > D || r0 < 0 || r0 > m || t < 0 || t > R || dxl < 0 || dxl > D || dqa < 0 || dqa > D) {
            if (threadIdx.x == 0) report_bad(A.err, 2, m, r0, t, dqa);
            return;
        }
    }
    double fl = 0.0;
    if (t > 0) {
        // rows r0.. of p: new = Vq^T old over the live columns of x; for the
        // diagonal block also columns r0..: new = old Vq
        const int dx = (x == p) ? m : live_rows(A, x, lane);
        T* slab = reinterpret_cast<T*>(rot_smem);
        T* vs = slab + (size_t)D * RC;
        const int mcol = (x == p) ? m : -1;
        rotate_block<T, NU>(B, D, tr, r0, R, dx, mcol, Vq, slab, vs);
        fl += 2.0 * R * (double)R * dx;
        if (x == p) fl += 2.0 * m * (double)R * R;
    }
    if (A.rowblk_fill[ci * A.nrow_max + b]) {   // drop the remaining redundant rows
        const int dq = A.dim[x * LN + lane];
        const int rows = m - (r0 + t);
        for (int e = threadIdx.x; e < rows * dq; e += NT) {
            int i = e / dq, j = e % dq;
            belem(B, D, tr, r0 + t + i, j) = 0.0;
        }
    }
    if (threadIdx.x == 0 && fl > 0.0) add_stats(A.stats, H2_KIND_ROTATE, fl, 8.0 * fl / R);
}
template <typename T, int NU>
__global__ void __launch_bounds__(NT) k_rotate(FactorArgs A) { k_rotate_body<T, NU>(A, blockIdx.x, blockIdx.y); }
template <typename T, int NU>
__global__ void __launch_bounds__(NT) k_rotate_g(GroupArgs<FactorArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_rotate_body<T, NU>(G.args[m], blockIdx.x - G.off[m], blockIdx.y);
}

// FP64 path: one output per thread and step over the exact R x nj outputs of
// each pass (no padded rows or columns: every DFMA is algorithmic)
__device__ __forceinline__ void k_rotate_fp64_body(const FactorArgs& A, const int bx, const int by) {
    HbScope hb_(2);
    const int ci = bx / A.nrow_max, b = bx % A.nrow_max, lane = by;
    if (lane >= *A.active || b >= A.nrow[ci]) return;
    extern __shared__ double tile[];          // R x RC
    const int D = A.D, LN = A.lanes;
    const int p = A.cl[ci];
    const double* scr = A.scratch + ((size_t)ci * LN + lane) * A.lay.total;
    const int* hdr = (const int*)(scr + A.lay.hdr);
    if (!hdr[4]) return;
    const int r0 = hdr[2], t = hdr[3];
    const int m = A.dim[p * LN + lane];
    const int R = m - r0;
    const double* Vq = scr + A.lay.vq;
    const int x = A.rowblk_other[ci * A.nrow_max + b];
    const int tr = A.rowblk_trans[ci * A.nrow_max + b];
    double* B = slot_ptr(A.slots, A.rowblk[ci * A.nrow_max + b], LN, lane, D);
    {
        const int dxl = live_rows(A, x, lane), dqa = A.dim[x * LN + lane];
        if (m < 0 || m > D || r0 < 0 || r0 > m || t < 0 || t > R || dxl < 0 || dxl > D || dqa < 0 || dqa > D) {
            if (threadIdx.x == 0) report_bad(A.err, 2, m, r0, t, dqa);
            return;
        }
    }
    double fl = 0.0;
    if (t > 0) {
        // rows r0.. of p: new = Vq^T old, over the live columns of x
        const int dx = (x == p) ? m : live_rows(A, x, lane);
        for (int j0 = 0; j0 < dx; j0 += RC) {
            const int nj = min(RC, dx - j0);
            for (int e = threadIdx.x; e < R * nj; e += NT) {
                int k = e / nj, j = e % nj;
                tile[k * RC + j] = belem(B, D, tr, r0 + k, j0 + j);
            }
            __syncthreads();
            for (int e = threadIdx.x; e < R * nj; e += NT) {
                int i = e / nj, j = e % nj;
                double v = 0.0;
                for (int k = 0; k < R; ++k) v += Vq[(size_t)k * D + i] * tile[k * RC + j];
                belem(B, D, tr, r0 + i, j0 + j) = v;
            }
            __syncthreads();
        }
        fl += 2.0 * R * (double)R * dx;
        if (x == p) {      // diagonal block: columns r0.. for every row
            for (int i0 = 0; i0 < m; i0 += RC) {
                const int ni = min(RC, m - i0);
                for (int e = threadIdx.x; e < ni * R; e += NT) {
                    int i = e / R, k = e % R;
                    tile[k * RC + i] = B[(size_t)(i0 + i) * D + r0 + k];
                }
                __syncthreads();
                for (int e = threadIdx.x; e < ni * R; e += NT) {
                    int i = e / R, j = e % R;
                    double v = 0.0;
                    for (int k = 0; k < R; ++k) v += tile[k * RC + i] * Vq[(size_t)k * D + j];
                    B[(size_t)(i0 + i) * D + r0 + j] = v;
                }
                __syncthreads();
            }
            fl += 2.0 * m * (double)R * R;
        }
    }
    if (A.rowblk_fill[ci * A.nrow_max + b]) {   // drop the remaining redundant rows
        const int dq = A.dim[x * LN + lane];
        const int rows = m - (r0 + t);
        for (int e = threadIdx.x; e < rows * dq; e += NT) {
            int i = e / dq, j = e % dq;
            belem(B, D, tr, r0 + t + i, j) = 0.0;
        }
    }
    if (threadIdx.x == 0 && fl > 0.0) add_stats(A.stats, H2_KIND_ROTATE, fl, 8.0 * fl / R);
}
__global__ void __launch_bounds__(NT) k_rotate_fp64(FactorArgs A) { k_rotate_fp64_body(A, blockIdx.x, blockIdx.y); }
__global__ void __launch_bounds__(NT) k_rotate_fp64_g(GroupArgs<FactorArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_rotate_fp64_body(G.args[m], blockIdx.x - G.off[m], blockIdx.y);
}

// FP64_TC rotation: the same products as k_rotate_fp64 (rows r0.. of the
// block become V^T old; for the diagonal block, columns r0.. become old V)
// from exact 7-bit digits on the tensor cores (see k_schur_oz).  V^T's digit
// planes come from the recompression kernel; the block's digits are taken for
// 32 columns (rows) at a time, all of them before any output of that chunk is
// written, so the update stays in place.
__host__ __device__ constexpr int oz_rpad(int D) { return (D + 31) / 32 * 32; }
__host__ __device__ constexpr size_t rotate_oz_smem(int D) {
    return (size_t)OZP * TS * (oz_rpad(D) + 8) * 2 + (size_t)OZP * TS * OZLD * 2 + TS * sizeof(int);
}

__device__ __forceinline__ void k_rotate_oz_body(const FactorArgs& A, const int bx, const int by) {
    HbScope hb_(2);
    const int ci = bx / A.nrow_max, b = bx % A.nrow_max, lane = by;
    if (lane >= *A.active || b >= A.nrow[ci]) return;
    extern __shared__ __align__(16) unsigned char rz_smem[];
    const int D = A.D, LN = A.lanes;
    const int p = A.cl[ci];
    const double* scr = A.scratch + ((size_t)ci * LN + lane) * A.lay.total;
    const int* hdr = (const int*)(scr + A.lay.hdr);
    if (!hdr[4]) return;
    const int r0 = hdr[2], t = hdr[3];
    const int m = A.dim[p * LN + lane];
    const int R = m - r0;
    const int x = A.rowblk_other[ci * A.nrow_max + b];
    const int tr = A.rowblk_trans[ci * A.nrow_max + b];
    double* B = slot_ptr(A.slots, A.rowblk[ci * A.nrow_max + b], LN, lane, D);
    {
        const int dxl = live_rows(A, x, lane), dqa = A.dim[x * LN + lane];
        if (m < 0 || m > D || r0 < 0 || r0 > m || t < 0 || t > R || dxl < 0 || dxl > D || dqa < 0 || dqa > D) {
            if (threadIdx.x == 0) report_bad(A.err, 2, m, r0, t, dqa);
            return;
        }
    }
    double fl = 0.0;
    if (t > 0) {
        const int dk = A.lay.dk, Rp32 = oz_rpad(R), LA = oz_rpad(D) + 8;
        const uint16_t* vd = reinterpret_cast<const uint16_t*>(scr + A.lay.vd);
        const int* ve = reinterpret_cast<const int*>(scr + A.lay.ve);
        uint16_t* sAll = reinterpret_cast<uint16_t*>(rz_smem);              // [OZP][TS][LA]: the block's digits
        uint16_t* sCh = sAll + (size_t)OZP * TS * LA;                        // [OZP][TS][OZLD]: V^T digits
        int* sExp = reinterpret_cast<int*>(sCh + (size_t)OZP * TS * OZLD);   // [TS]
        const int w = threadIdx.x / 32, l = threadIdx.x % 32, gid = l / 4, tig = l % 4;
        const int mi = w / 4, ni = w % 4;
        // copy rows v0.. of V^T's planes, k0.. (32 x 32) into sCh
        auto copy_vt = [&](int v0, int nrow, int k0) {
            for (int e = threadIdx.x; e < OZP * TS * 4; e += NT) {
                const int pp = e / (TS * 4), r = (e / 4) % TS, c = e % 4;
                int4 v = make_int4(0, 0, 0, 0);
                if (r < nrow) v = *reinterpret_cast<const int4*>(&vd[((size_t)pp * D + v0 + r) * dk + k0 + 8 * c]);
                *reinterpret_cast<int4*>(&sCh[((size_t)pp * TS + r) * OZLD + 8 * c]) = v;
            }
        };
        // digits of 32 vectors of R values (vector jj, entry k) = get(jj, k), with
        // each vector's largest exponent, into sAll / sExp
        auto take = [&](int nvec, auto get) {
            for (int jj = w; jj < TS; jj += NT / 32) {
                int e = 0;
                if (jj < nvec)
                    for (int k = l; k < R; k += 32) e = max(e, oz_expo(get(jj, k)));
                for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
                if (l == 0) sExp[jj] = e;
            }
            __syncthreads();
            const int npair = Rp32 / 2;
            for (int e = threadIdx.x; e < TS * npair; e += NT) {
                const int jj = e / npair, k = 2 * (e % npair);
                const double x0 = (jj < nvec && k < R) ? get(jj, k) : 0.0;
                const double x1 = (jj < nvec && k + 1 < R) ? get(jj, k + 1) : 0.0;
                uint32_t d0[OZP], d1[OZP];
                oz_digits(x0, sExp[jj], d0);
                oz_digits(x1, sExp[jj], d1);
#pragma unroll
                for (int pp = 0; pp < OZP; ++pp)
                    *reinterpret_cast<uint32_t*>(&sAll[((size_t)pp * TS + jj) * LA + k]) = d0[pp] | (d1[pp] << 16);
            }
            __syncthreads();
        };
        // row side: rows r0 + i (i < R), columns j0.. of the dx live columns of x
        const int dx = (x == p) ? m : live_rows(A, x, lane);
        for (int j0 = 0; j0 < dx; j0 += TS) {
            const int nj = min(TS, dx - j0);
            take(nj, [&](int jj, int k) { return belem(B, D, tr, r0 + k, j0 + jj); });
            for (int i0 = 0; i0 < R; i0 += TS) {
                const int nr = min(TS, R - i0);
                const bool act = 16 * mi < nr && 8 * ni < nj;
                long long hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
                for (int k0 = 0; k0 < R; k0 += OZK) {
                    copy_vt(i0, nr, k0);
                    __syncthreads();
                    if (act)
                        oz_warp_chunk(sCh, TS * OZLD, OZLD, sAll + k0, TS * LA, LA, mi, ni, min(OZK, R - k0), hi, lo);
                    __syncthreads();
                }
                if (act)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int r = 16 * mi + gid + (c >= 2 ? 8 : 0), q = 8 * ni + 2 * tig + (c & 1);
                        if (r < nr && q < nj)
                            belem(B, D, tr, r0 + i0 + r, j0 + q) = oz_value(hi[c], lo[c], ve[i0 + r], sExp[q]);
                    }
            }
            __syncthreads();
        }
        fl += 2.0 * R * (double)R * dx;
        if (x == p) {   // column side: columns r0.. of every row, new = old V
            for (int i0 = 0; i0 < m; i0 += TS) {
                const int nr = min(TS, m - i0);
                take(nr, [&](int ii, int k) { return B[(size_t)(i0 + ii) * D + r0 + k]; });
                for (int j0 = 0; j0 < R; j0 += TS) {
                    const int nc = min(TS, R - j0);
                    const bool act = 16 * mi < nr && 8 * ni < nc;
                    long long hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
                    for (int k0 = 0; k0 < R; k0 += OZK) {
                        copy_vt(j0, nc, k0);
                        __syncthreads();
                        if (act)
                            oz_warp_chunk(sAll + k0, TS * LA, LA, sCh, TS * OZLD, OZLD, mi, ni, min(OZK, R - k0), hi,
                                          lo);
                        __syncthreads();
                    }
                    if (act)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int r = 16 * mi + gid + (c >= 2 ? 8 : 0), q = 8 * ni + 2 * tig + (c & 1);
                            if (r < nr && q < nc)
                                B[(size_t)(i0 + r) * D + r0 + j0 + q] = oz_value(hi[c], lo[c], sExp[r], ve[j0 + q]);
                        }
                }
                __syncthreads();
            }
            fl += 2.0 * m * (double)R * R;
        }
    }
    if (A.rowblk_fill[ci * A.nrow_max + b]) {   // drop the remaining redundant rows
        const int dq = A.dim[x * LN + lane];
        const int rows = m - (r0 + t);
        for (int e = threadIdx.x; e < rows * dq; e += NT) {
            int i = e / dq, j = e % dq;
            belem(B, D, tr, r0 + t + i, j) = 0.0;
        }
    }
    if (threadIdx.x == 0 && fl > 0.0) add_stats(A.stats, H2_KIND_ROTATE, fl, 8.0 * fl / R);
}
__global__ void __launch_bounds__(NT) k_rotate_oz(FactorArgs A) { k_rotate_oz_body(A, blockIdx.x, blockIdx.y); }
__global__ void __launch_bounds__(NT) k_rotate_oz_g(GroupArgs<FactorArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_rotate_oz_body(G.args[m], blockIdx.x - G.off[m], blockIdx.y);
}

// ---- (iii) Bunch-Kaufman LDL^T of S_pp^RR (Eq. blr2-diag-ldl) and its
// negative-pivot count: one CTA per (cluster, lane)
template <int NTH>
__device__ __forceinline__ void k_ldl_body(const FactorArgs& A, const int use_smem, const int bx, const int by) {
    HbScope hb_(3);
    const int ci = bx, lane = by;
    if (lane >= *A.active) return;
    extern __shared__ double sF[];
    __shared__ unsigned long long rkey[2 * NTH / 32];
    __shared__ int ridx[2 * NTH / 32];
    __shared__ int s_neg, s_bad;
    __shared__ double s_mp;
    const int D = A.D, LN = A.lanes;
    const int p = A.cl[ci];
    const int m = A.dim[p * LN + lane], rk1 = A.rk[p * LN + lane];
    const int Rp = m - rk1;
    double* scr = A.scratch + ((size_t)ci * LN + lane) * A.lay.total;
    int* hdr = (int*)(scr + A.lay.hdr);
    if (m < 0 || m > D || rk1 < 0 || rk1 > m) {
        if (threadIdx.x == 0) {
            hdr[0] = 0;
            hdr[1] = 0;     // later kernels of this elimination skip it
            report_bad(A.err, 3, m, rk1, D, 0);
        }
        return;
    }
    if (threadIdx.x == 0) {
        hdr[0] = rk1;
        hdr[1] = Rp;
        s_neg = 0;
        s_bad = 0;
        s_mp = 1.0 / 0.0;
    }
    if (Rp <= 0) return;
    double* F = scr + A.lay.f;
    int* perm = (int*)(scr + A.lay.iperm);
    int* piv = perm + D;
    const double* Bpp = slot_ptr(A.slots, A.targ_slot[ci * A.ntarg_max], LN, lane, D);   // target 0 = p
    double* S = use_smem ? sF : F;
    // odd leading dimension in shared memory (conflict-free column reads)
    const int lds = use_smem ? (Rp | 1) : D;
    double* bkbuf = use_smem ? sF + (size_t)Rp * lds : scr + A.lay.tmp;   // 4 Rp <= D*D doubles
    for (int e = threadIdx.x; e < Rp * Rp; e += NTH) {      // lower triangle and diagonal
        int i = e / Rp, j = e % Rp;
        if (j <= i) S[(size_t)i * lds + j] = Bpp[(size_t)(rk1 + i) * D + rk1 + j];
    }
    __syncthreads();
    cta_bk_ldl_lower<NTH>(S, lds, Rp, perm, piv, rkey, ridx, &s_neg, &s_mp, &s_bad, A.zero_pivot, bkbuf);
    if (use_smem)
        for (int e = threadIdx.x; e < Rp * Rp; e += NTH) {
            int i = e / Rp, j = e % Rp;
            if (j <= i) F[(size_t)i * D + j] = S[(size_t)i * lds + j];
        }
    if (threadIdx.x == 0) {
        atomicAdd(&A.neg[lane], (unsigned long long)s_neg);
        double mp = s_mp;
        if (!(mp >= 0.0)) mp = 0.0;
        atomicMin(&A.minpiv[lane], (unsigned long long)__double_as_longlong(mp));
        if (s_bad) atomicOr(A.err, 1);
        add_stats(A.stats, H2_KIND_LDL, (double)Rp * Rp * Rp / 3.0, 16.0 * (double)Rp * Rp);
    }
}
template <int NTH>
__global__ void __launch_bounds__(NTH) k_ldl(FactorArgs A, int use_smem) { k_ldl_body<NTH>(A, use_smem, blockIdx.x, blockIdx.y); }
template <int NTH>
__global__ void __launch_bounds__(NTH) k_ldl_g(GroupArgs<FactorArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_ldl_body<NTH>(G.args[m], G.flag[m], blockIdx.x - G.off[m], blockIdx.y);
}

// The same step with one warp per (cluster, lane) block, LW blocks per CTA
// (blocks of dimension <= 64): warp w of CTA bx takes item bx * LW + w of the
// colour's ncl * lanes items, its block staged in its own shared-memory slice.
constexpr int LW = 2;
__host__ __device__ constexpr size_t ldl_warp_slice(int D) { return (size_t)D * D + 4 * (size_t)D; }
__device__ __forceinline__ void k_ldl_warp_body(const FactorArgs& A, const int bx) {
    HbScope hb_(3);
    const int w = threadIdx.x / 32, l32 = threadIdx.x % 32;
    const int LN = A.lanes, D = A.D;
    const int item = bx * LW + w;
    if (item >= A.ncl * LN) return;
    const int ci = item % A.ncl, lane = item / A.ncl;
    if (lane >= *A.active) return;
    extern __shared__ double sW[];
    double* S = sW + (size_t)w * ldl_warp_slice(D);
    const int p = A.cl[ci];
    const int m = A.dim[p * LN + lane], rk1 = A.rk[p * LN + lane];
    const int Rp = m - rk1;
    double* scr = A.scratch + ((size_t)ci * LN + lane) * A.lay.total;
    int* hdr = (int*)(scr + A.lay.hdr);
    if (m < 0 || m > D || rk1 < 0 || rk1 > m) {
        if (l32 == 0) {
            hdr[0] = 0;
            hdr[1] = 0;
            report_bad(A.err, 3, m, rk1, D, 0);
        }
        return;
    }
    if (l32 == 0) {
        hdr[0] = rk1;
        hdr[1] = Rp;
    }
    if (Rp <= 0) return;
    double* F = scr + A.lay.f;
    int* perm = (int*)(scr + A.lay.iperm);
    int* piv = perm + D;
    const double* Bpp = slot_ptr(A.slots, A.targ_slot[ci * A.ntarg_max], LN, lane, D);   // target 0 = p
    for (int e = l32; e < Rp * Rp; e += 32) {
        int i = e / Rp, j = e % Rp;
        S[(size_t)i * Rp + j] = Bpp[(size_t)(rk1 + i) * D + rk1 + j];
    }
    __syncwarp();
    int neg = 0, bad = 0;
    double mp = 1.0 / 0.0;
    warp_bk_ldl(S, Rp, Rp, perm, piv, &neg, &mp, &bad, A.zero_pivot, S + (size_t)Rp * Rp);
    for (int e = l32; e < Rp * Rp; e += 32) {
        int i = e / Rp, j = e % Rp;
        F[(size_t)i * D + j] = S[(size_t)i * Rp + j];
    }
    if (l32 == 0) {
        atomicAdd(&A.neg[lane], (unsigned long long)neg);
        if (!(mp >= 0.0)) mp = 0.0;
        atomicMin(&A.minpiv[lane], (unsigned long long)__double_as_longlong(mp));
        if (bad) atomicOr(A.err, 1);
        add_stats(A.stats, H2_KIND_LDL, (double)Rp * Rp * Rp / 3.0, 16.0 * (double)Rp * Rp);
    }
}
__global__ void __launch_bounds__(32 * LW) k_ldl_warp(FactorArgs A) { k_ldl_warp_body(A, blockIdx.x); }
__global__ void __launch_bounds__(32 * LW) k_ldl_warp_g(GroupArgs<FactorArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_ldl_warp_body(G.args[m], blockIdx.x - G.off[m]);
}


// ---- (iv) W_a = S_ap^{.R} P L^{-T}, Y_a = W_a D^{-1} (Eq. blr2-diag-elimination):
// one CTA per (target, cluster, lane); column-blocked forward substitution
// (JB columns per block: a parallel update from the solved columns, then a
// short per-row solve inside the block)
constexpr int JB = 8;
// T is the arithmetic of the solve and the type W and Y are stored in: double
// (FP64 path) or float (mixed path: the FP64 factor L, D of the LDL step is
// rounded to FP32, as are the products that form the Schur update)
// 1 / d_j for a 1x1 pivot at j, 1 / det for a 2x2 pivot starting at j (0
// elsewhere), from the factor's entries rounded to T: Y = W D^-1 then
// multiplies by it instead of dividing once per element
template <typename T>
__device__ __forceinline__ T pivot_reciprocal(const double* F, int D, int Rp, const int* piv, int j) {
    const int pv = piv[j];
    const bool two = pv == 2 && j + 1 < Rp;
    if (pv != 1 && !two) return (T)0;
    T x = (T)F[(size_t)j * D + j];
    if (two) {
        const T b0 = (T)F[(size_t)(j + 1) * D + j], c0 = (T)F[(size_t)(j + 1) * D + j + 1];
        x = x * c0 - b0 * b0;
    }
    return (T)1 / x;
}

template <typename T>
__device__ __forceinline__ void k_trsm_body(const FactorArgs& A, const int use_smem, const int bx, const int by) {
    HbScope hb_(4);
    const int ci = bx / A.ntarg_max, ti = bx % A.ntarg_max, lane = by;
    if (lane >= *A.active || ti >= A.ntarg[ci]) return;
    extern __shared__ double sh[];
    const int D = A.D, LN = A.lanes;
    const int p = A.cl[ci];
    double* scr = A.scratch + ((size_t)ci * LN + lane) * A.lay.total;
    int* hdr = (int*)(scr + A.lay.hdr);
    const int rk1 = hdr[0], Rp = hdr[1];
    if (Rp <= 0) return;
    const int a = A.targ[ci * A.ntarg_max + ti];
    const int rows = (a == p) ? rk1 : live_rows(A, a, lane);
    if (Rp > D || rk1 < 0 || rk1 + Rp > D || rows < 0 || rows > D) {
        if (threadIdx.x == 0) {
            hdr[HDR_ROWS + ti] = 0;
            report_bad(A.err, 4, rk1, Rp, rows, a);
        }
        return;
    }
    if (threadIdx.x == 0) {
        hdr[HDR_ROWS + ti] = rows;
        double fs = 0.0, bs = 0.0;
        for (int tj = 0; tj <= ti; ++tj) {
            int b2 = A.targ[ci * A.ntarg_max + tj];
            double rb = (b2 == p) ? rk1 : live_rows(A, b2, lane);
            // a diagonal block: its lower triangle (DFMA kernel) or the tiles
            // on and below the tile diagonal (FP32 and digit kernels)
            const double ent = tj != ti ? rows * rb
                             : (sizeof(T) == 8 && A.lay.dk == 0) ? 0.5 * rows * (rows + 1.0)
                                                                 : lower_tile_entries(rows, sizeof(T) == 4 ? TSF : TS);
            fs += 2.0 * ent * Rp;
            bs += 8.0 * (rows * (double)Rp + rb * Rp + 2.0 * rows * rb);
        }
        add_stats(A.stats, H2_KIND_SCHUR, fs, bs);
        add_stats(A.stats, H2_KIND_TRSM, (double)rows * Rp * Rp + (double)rows * Rp,
                  8.0 * 3.0 * rows * (double)Rp);
    }
    if (rows <= 0) return;
    const int tr = A.targ_trans[ci * A.ntarg_max + ti];
    const double* B = slot_ptr(A.slots, A.targ_slot[ci * A.ntarg_max + ti], LN, lane, D);
    T* W = reinterpret_cast<T*>(scr + A.lay.w + (size_t)ti * D * D);
    T* Y = reinterpret_cast<T*>(scr + A.lay.y + (size_t)ti * D * D);
    if (use_smem == 2) {
        // everything in shared memory: L with the (k+1, k) entries of 2x2
        // pivots read as 0 (they hold D's off-diagonal), D's diagonal and
        // off-diagonal apart, and W; the same expressions as the path below
        const double* F = scr + A.lay.f;
        const int* perm = (const int*)(scr + A.lay.iperm);
        const int* piv = perm + D;
        // rows of L and of W padded to Rp + 1 values: the update loop reads
        // L(j, k) for 8 consecutive j in one warp, which a stride of Rp (a
        // multiple of 16 at these levels) would put in one bank
        const int ldl = Rp + 1;
        T* sLz = reinterpret_cast<T*>(sh);                       // Rp x (Rp + 1)
        T* sWm = sLz + (size_t)Rp * ldl;                         // rows x (Rp + 1)
        T* sDg = sWm + (size_t)rows * (Rp + 1);
        T* sOd = sDg + Rp;
        T* sRc = sOd + Rp;      // 1 / d of a 1x1 pivot, 1 / det at the first column of a 2x2
        int* sPerm = reinterpret_cast<int*>(sRc + Rp);
        int* sPiv = sPerm + Rp;
        const int ldw = Rp + 1;
        for (int e = threadIdx.x; e < Rp * Rp; e += NT) {
            const int j = e / Rp, k = e % Rp;
            sLz[j * ldl + k] = (k < j && !(piv[k] == 2 && j == k + 1)) ? (T)F[(size_t)j * D + k] : (T)0;
        }
        for (int j = threadIdx.x; j < Rp; j += NT) {
            const T dj = (T)F[(size_t)j * D + j];
            sDg[j] = dj;
            sOd[j] = (piv[j] == 2 && j + 1 < Rp) ? (T)F[(size_t)(j + 1) * D + j] : (T)0;
            sRc[j] = pivot_reciprocal<T>(F, D, Rp, piv, j);
            sPerm[j] = perm[j];
            sPiv[j] = piv[j];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * Rp; e += NT) {      // W = S_ap^{.R} P
            // consecutive threads read consecutive addresses of the stored block
            const int i = tr ? e % rows : e / Rp, j = tr ? e / rows : e % Rp;
            sWm[i * ldw + j] = (T)(tr ? B[(size_t)(rk1 + sPerm[j]) * D + i] : B[(size_t)i * D + rk1 + sPerm[j]]);
        }
        __syncthreads();
        for (int jb = 0; jb < Rp; jb += JB) {
            const int nb = min(JB, Rp - jb);
            if (jb > 0) {
                for (int e = threadIdx.x; e < rows * nb; e += NT) {
                    const int i = e / nb, j = jb + e % nb;
                    const T* wi = sWm + i * ldw;
                    const T* lj = sLz + (size_t)j * ldl;
                    T v = wi[j];
                    for (int k = 0; k < jb; ++k) v -= wi[k] * lj[k];
                    sWm[i * ldw + j] = v;
                }
                __syncthreads();
            }
            for (int i = threadIdx.x; i < rows; i += NT) {
                T* wi = sWm + i * ldw;
                for (int j = jb + 1; j < jb + nb; ++j) {
                    const T* lj = sLz + (size_t)j * ldl;
                    T v = wi[j];
                    for (int k = jb; k < j; ++k) v -= wi[k] * lj[k];
                    wi[j] = v;
                }
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < rows * Rp; e += NT) {       // Y = W D^{-1}
            const int i = e / Rp, j = e % Rp;
            const T* wi = sWm + i * ldw;
            T v;
            if (sPiv[j] == 1) {
                v = wi[j] * sRc[j];
            } else {
                const int j0 = sPiv[j] == 2 ? j : j - 1;
                const T b0 = sOd[j0], c0 = sDg[j0 + 1], a0 = sDg[j0];
                const T idet = sRc[j0];
                const T w0 = wi[j0], w1 = wi[j0 + 1];
                v = (j == j0) ? (w0 * c0 - w1 * b0) * idet : (w1 * a0 - w0 * b0) * idet;
            }
            Y[(size_t)i * D + j] = v;
            W[(size_t)i * D + j] = wi[j];
        }
    } else {
        // L, D and the pivots: staged in shared memory (as T) when they fit
        const double* F = scr + A.lay.f;
        const int* perm = (const int*)(scr + A.lay.iperm);
        const int* piv = perm + D;
        const T* sL = nullptr;
        const int* sperm = perm;
        const int* spiv = piv;
        const int ldl = Rp + 1;                                      // padded as in the path above
        T* sRc = reinterpret_cast<T*>(sh);                           // Rp pivot reciprocals
        for (int j = threadIdx.x; j < Rp; j += NT) sRc[j] = pivot_reciprocal<T>(F, D, Rp, piv, j);
        if (use_smem) {
            T* L2 = sRc + Rp;                                        // Rp x (Rp + 1)
            int* p2 = reinterpret_cast<int*>(L2 + (size_t)Rp * ldl);
            int* v2 = p2 + Rp;
            for (int e = threadIdx.x; e < Rp * Rp; e += NT) L2[(e / Rp) * ldl + e % Rp] = (T)F[(size_t)(e / Rp) * D + e % Rp];
            for (int e = threadIdx.x; e < Rp; e += NT) { p2[e] = perm[e]; v2[e] = piv[e]; }
            sL = L2;
            sperm = p2;
            spiv = v2;
        }
        __syncthreads();
        auto Fx = [&](int j, int k) -> T {  // entry (j, k) of the packed factor
            return use_smem ? sL[(size_t)j * ldl + k] : (T)F[(size_t)j * D + k];
        };
        auto Lx = [&](int j, int k) -> T {  // L(j, k), k < j, of the unit lower factor
            return (spiv[k] == 2 && j == k + 1) ? (T)0 : Fx(j, k);
        };
        for (int e = threadIdx.x; e < rows * Rp; e += NT) {       // W = S_ap^{.R} P
            int i = e / Rp, j = e % Rp;
            W[(size_t)i * D + j] = (T)(tr ? B[(size_t)(rk1 + sperm[j]) * D + i] : B[(size_t)i * D + rk1 + sperm[j]]);
        }
        __syncthreads();
        for (int jb = 0; jb < Rp; jb += JB) {
            const int nb = min(JB, Rp - jb);
            if (jb > 0) {
                for (int e = threadIdx.x; e < rows * nb; e += NT) {
                    int i = e / nb, j = jb + e % nb;
                    T v = W[(size_t)i * D + j];
                    const T* wi = W + (size_t)i * D;
                    for (int k = 0; k < jb; ++k) v -= wi[k] * Lx(j, k);
                    W[(size_t)i * D + j] = v;
                }
                __syncthreads();
            }
            for (int i = threadIdx.x; i < rows; i += NT) {
                T* wi = W + (size_t)i * D;
                for (int j = jb + 1; j < jb + nb; ++j) {
                    T v = wi[j];
                    for (int k = jb; k < j; ++k) v -= wi[k] * Lx(j, k);
                    wi[j] = v;
                }
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < rows * Rp; e += NT) {       // Y = W D^{-1}
            int i = e / Rp, j = e % Rp;
            const T* wi = W + (size_t)i * D;
            T v;
            if (spiv[j] == 1) {
                v = wi[j] * sRc[j];
            } else {
                int j0 = spiv[j] == 2 ? j : j - 1;
                T a0 = Fx(j0, j0), b0 = Fx(j0 + 1, j0), c0 = Fx(j0 + 1, j0 + 1);
                T idet = sRc[j0];
                T w0 = wi[j0], w1 = wi[j0 + 1];
                v = (j == j0) ? (w0 * c0 - w1 * b0) * idet : (w1 * a0 - w0 * b0) * idet;
            }
            Y[(size_t)i * D + j] = v;
        }
    }
    if (A.lay.dk > 0) {          // FP64_TC: digit planes of W_a and Y_a, once
        __syncthreads();
        const int dk = A.lay.dk;
        uint16_t* wd = reinterpret_cast<uint16_t*>(scr + A.lay.wd) + (size_t)ti * OZP * D * dk;
        uint16_t* yd = reinterpret_cast<uint16_t*>(scr + A.lay.yd) + (size_t)ti * OZP * D * dk;
        int* we = reinterpret_cast<int*>(scr + A.lay.we) + ti * D;
        int* ye = reinterpret_cast<int*>(scr + A.lay.ye) + ti * D;
        const int w = threadIdx.x / 32, l = threadIdx.x % 32;
        for (int r = w; r < rows; r += NT / 32) {
            int ea = 0, eb = 0;
            for (int k = l; k < Rp; k += 32) {
                ea = max(ea, oz_expo((double)W[(size_t)r * D + k]));
                eb = max(eb, oz_expo((double)Y[(size_t)r * D + k]));
            }
            for (int o = 16; o > 0; o >>= 1) {
                ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, o));
                eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, o));
            }
            if (l == 0) { we[r] = ea; ye[r] = eb; }
        }
        __syncthreads();
        const int npair = (Rp + 31) / 32 * 16;       // k pairs up to the padded width
        for (int e = threadIdx.x; e < 2 * rows * npair; e += NT) {
            const int op = e / (rows * npair), rem = e % (rows * npair);
            const int r = rem / npair, k = 2 * (rem % npair);
            const T* src = op ? Y : W;
            const int em = op ? ye[r] : we[r];
            const double x0 = k < Rp ? (double)src[(size_t)r * D + k] : 0.0;
            const double x1 = k + 1 < Rp ? (double)src[(size_t)r * D + k + 1] : 0.0;
            uint32_t d0[OZP], d1[OZP];
            oz_digits(x0, em, d0);
            oz_digits(x1, em, d1);
            uint16_t* dst = op ? yd : wd;
#pragma unroll
            for (int p = 0; p < OZP; ++p)
                *reinterpret_cast<uint32_t*>(&dst[((size_t)p * D + r) * dk + k]) = d0[p] | (d1[p] << 16);
        }
    }
}
template <typename T>
__global__ void __launch_bounds__(NT) k_trsm(FactorArgs A, int use_smem) { k_trsm_body<T>(A, use_smem, blockIdx.x, blockIdx.y); }
template <typename T>
__global__ void __launch_bounds__(NT) k_trsm_g(GroupArgs<FactorArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_trsm_body<T>(G.args[m], G.flag[m], blockIdx.x - G.off[m], blockIdx.y);
}

struct SchurArgs {
    double* slots;
    int D, lanes;
    const SchurPair* pairs;
    int tiles_per_pair, tdim;
    const double* scratch;
    ScratchLayout lay;
    const int* active;
    int* err;
    const int* ntarg;   // targets of each elimination of the colour (tcgen05 kernel)
    int npanel;         // 128-row panels per elimination (tcgen05 kernel)
};

// S_ab[i0:i0+32, j0:j0+32] -= W_a Y_b^T (Eq. blr2-diag-schur).  T is the
// arithmetic of the products and the type k_trsm stored W, Y in: double (FP64
// path) or float (mixed path: FP32 products and accumulation, the FP64 block
// updated by the rounded result).
// NU rows (ty + 8u, u < NU) of the tile against column tx over kc values of k
template <typename T, int NU>
__device__ __forceinline__ void schur_rows(const T (*sR)[TS + 1], const T (*sC)[TS + 1], int kc, int tx, int ty,
                                           T (&acc)[4]) {
#pragma unroll 8
    for (int k = 0; k < kc; ++k) {
        const T y = sC[tx][k];
#pragma unroll
        for (int u = 0; u < NU; ++u) acc[u] += sR[ty + 8 * u][k] * y;
    }
}

// Diagonal tile (i0, i0) of a symmetric update S_aa -= W_a Y_a^T: only its
// nr (nr + 1) / 2 entries on and below the diagonal are computed (up to three
// per thread, the rows of W and of Y staged in sR / sC as for a full tile,
// each entry summed over k in the same order), and each is written to (r, c)
// and (c, r).  Entry t of the lower triangle is (r, c), t = r (r + 1) / 2 + c.
__device__ __forceinline__ void tri_index(int t, int& r, int& c) {
    r = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r > 0 && r * (r + 1) / 2 > t) --r;
    c = t - r * (r + 1) / 2;
}
template <typename T>
__device__ __forceinline__ void schur_diag_tile(double* B, int D, int trans, const T* W, const T* Y, int i0, int nr,
                                                int Rp, T (*sR)[TS + 1], T (*sC)[TS + 1]) {
    const int ne = nr * (nr + 1) / 2;
    T acc[3] = {0, 0, 0};
    for (int k0 = 0; k0 < Rp; k0 += TS) {
        const int kc = min(TS, Rp - k0);
        for (int e = threadIdx.x; e < TS * TS; e += NT) {
            const int r = e / TS, k = e % TS;
            sR[r][k] = (r < nr && k < kc) ? W[(size_t)(i0 + r) * D + k0 + k] : (T)0;
            sC[r][k] = (r < nr && k < kc) ? Y[(size_t)(i0 + r) * D + k0 + k] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int t = threadIdx.x + NT * u;
            if (t < ne) {
                int r, c;
                tri_index(t, r, c);
                T a = acc[u];
#pragma unroll 8
                for (int k = 0; k < kc; ++k) a += sR[r][k] * sC[c][k];
                acc[u] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        const int t = threadIdx.x + NT * u;
        if (t < ne) {
            int r, c;
            tri_index(t, r, c);
            belem(B, D, trans, i0 + r, i0 + c) -= (double)acc[u];
            if (c != r) belem(B, D, trans, i0 + c, i0 + r) -= (double)acc[u];
        }
    }
}

template <typename T>
__device__ __forceinline__ void k_schur_body(const SchurArgs& A, const int bx, const int by) {
    HbScope hb_(5);
    const int lane = by;
    if (lane >= *A.active) return;
    const int pi = bx / A.tiles_per_pair, tile = bx % A.tiles_per_pair;
    const SchurPair P = A.pairs[pi];
    const int D = A.D;
    const double* scr = A.scratch + ((size_t)P.elim * A.lanes + lane) * A.lay.total;
    const int* hdr = (const int*)(scr + A.lay.hdr);
    const int Rp = hdr[1];
    if (Rp <= 0) return;
    const int ra = hdr[HDR_ROWS + P.ta], rb = hdr[HDR_ROWS + P.tb];
    if (Rp > D || ra < 0 || ra > D || rb < 0 || rb > D) {
        if (threadIdx.x == 0 && tile == 0) report_bad(A.err, 5, Rp, ra, rb, D);
        return;
    }
    const int i0 = (tile / A.tdim) * TS, j0 = (tile % A.tdim) * TS;
    if (i0 >= ra || j0 >= rb) return;
    if (P.ta == P.tb && j0 > i0) return;           // written by the mirror of tile (j0, i0)
    __shared__ T sR[TS][TS + 1], sC[TS][TS + 1];
    if (P.ta == P.tb && j0 == i0) {                // its lower triangle only
        schur_diag_tile<T>(slot_ptr(A.slots, P.slot, A.lanes, lane, D), D, P.trans,
                           reinterpret_cast<const T*>(scr + A.lay.w + (size_t)P.ta * D * D),
                           reinterpret_cast<const T*>(scr + A.lay.y + (size_t)P.tb * D * D), i0,
                           min(TS, ra - i0), Rp, sR, sC);
        return;
    }
    // kept in shared memory, not in a register through the k loop (the
    // loop's first barrier publishes it)
    __shared__ int s_mirror;
    if (threadIdx.x == 0) s_mirror = P.ta == P.tb && j0 < i0;
    const T* W = reinterpret_cast<const T*>(scr + A.lay.w + (size_t)P.ta * D * D);
    const T* Y = reinterpret_cast<const T*>(scr + A.lay.y + (size_t)P.tb * D * D);
    // A warp owns the rows ty + 8u of the tile: rows past the block are not
    // computed (one warp-uniform choice among four unrolled loops, made once).
    // Padded columns sit in the lanes and cost as much as real ones, so the
    // tile is computed transposed when its columns are the more ragged side.
    const int nr = min(TS, ra - i0), nc = min(TS, rb - j0);
    const bool tp = nc < nr;
    const T* Rm = tp ? Y + (size_t)j0 * D : W + (size_t)i0 * D;    // row operand
    const T* Cm = tp ? W + (size_t)i0 * D : Y + (size_t)j0 * D;    // column operand
    const int nrow = tp ? nc : nr, ncol = tp ? nr : nc;
    const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;   // ty in 0..7
    const int nu = max(0, min(4, (nrow - ty + 7) / 8));
    T acc[4] = {0, 0, 0, 0};
    for (int k0 = 0; k0 < Rp; k0 += TS) {
        const int kc = min(TS, Rp - k0);
        for (int e = threadIdx.x; e < TS * TS; e += NT) {
            int r = e / TS, k = e % TS;
            sR[r][k] = (r < nrow && k < kc) ? Rm[(size_t)r * D + k0 + k] : (T)0;
            sC[r][k] = (r < ncol && k < kc) ? Cm[(size_t)r * D + k0 + k] : (T)0;
        }
        __syncthreads();
        switch (nu) {
            case 4: schur_rows<T, 4>(sR, sC, kc, tx, ty, acc); break;
            case 3: schur_rows<T, 3>(sR, sC, kc, tx, ty, acc); break;
            case 2: schur_rows<T, 2>(sR, sC, kc, tx, ty, acc); break;
            case 1: schur_rows<T, 1>(sR, sC, kc, tx, ty, acc); break;
            default: break;
        }
        __syncthreads();
    }
    const bool mirror = s_mirror;
    double* B = slot_ptr(A.slots, P.slot, A.lanes, lane, D);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = ty + 8 * u;
        if (r < nrow && tx < ncol) {
            const int i = tp ? i0 + tx : i0 + r, j = tp ? j0 + r : j0 + tx;
            belem(B, D, P.trans, i, j) -= (double)acc[u];
            if (mirror) sR[i - i0][j - j0] = acc[u];   // the k loop ended with a barrier
        }
    }
    if (mirror) {
        __syncthreads();
        schur_mirror(B, D, P.trans, i0, j0, tp ? ncol : nrow, tp ? nrow : ncol, &sR[0][0], TS + 1, TS);
    }
}
// 8 CTAs of 256 threads per SM (32 registers): the FP64 pipe stays fed from
// shared memory at full occupancy
template <typename T>
__global__ void __launch_bounds__(NT, 8) k_schur(SchurArgs A) { k_schur_body<T>(A, blockIdx.x, blockIdx.y); }
template <typename T>
__global__ void __launch_bounds__(NT) k_schur_g(GroupArgs<SchurArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_schur_body<T>(G.args[m], blockIdx.x - G.off[m], blockIdx.y);
}

// FP64-accurate Schur products on the tensor cores (precision H2_PREC_FP64_TC).
// Every row of W (and of Y) is scaled by 2^e with |x| < 2^e over the row and
// cut into OZP = 8 signed 7-bit integer digits taken from the 53-bit
// significand: x = sign * 2^e * sum_p d_p 2^(-7p), d_p in [0, 127], exact up to
// the truncated bits below 2^(e-56).  Digits are exact in BF16, so
//   sum_k W_ik Y_jk = 2^(e_i + f_j) sum_t 2^(-7t) L_t,
//   L_t = sum_{p+q=t} sum_k d_p(W_ik) d_q(Y_jk),
// and the terms with t = p + q > 9 are dropped (each below 2^-56 of the
// row-scale product 2^(e_i + f_j)): 36 of the 64 digit pairs remain.  With the
// truncated bits of both operands, the error of a product of K terms stays
// below 2^-53 of the result plus 1.24e-16 K 2^(e_i + f_j).  Over a chunk of OZK = 32 values of k,
// |L_t| <= 8 * 32 * 127^2 < 2^22, and every partial sum an MMA forms is an
// integer below 2^24: BF16 products with FP32 accumulation (mma.sync
// m16n8k16) are exact.  Per chunk the level sums are folded into two exact
// int64 accumulators, hi = sum_{t=2..5} L_t 2^(7(5-t)) and lo = sum_{t=6..9}
// L_t 2^(7(9-t)); the product is rounded to FP64 once, from
// hi 2^-35 + lo 2^-63.  (Splitting FP64 operands into small-integer slices
// whose products a low-precision unit sums exactly is the scheme of Ozaki,
// Ogita, Oishi and Rump, 2012.)
__device__ __forceinline__ void k_schur_oz_body(const SchurArgs& A, const int bx, const int by) {
    HbScope hb_(5);
    const int lane = by;
    if (lane >= *A.active) return;
    const int pi = bx / A.tiles_per_pair, tile = bx % A.tiles_per_pair;
    const SchurPair P = A.pairs[pi];
    const int D = A.D;
    const double* scr = A.scratch + ((size_t)P.elim * A.lanes + lane) * A.lay.total;
    const int* hdr = (const int*)(scr + A.lay.hdr);
    const int Rp = hdr[1];
    if (Rp <= 0) return;
    const int ra = hdr[HDR_ROWS + P.ta], rb = hdr[HDR_ROWS + P.tb];
    if (Rp > D || ra < 0 || ra > D || rb < 0 || rb > D) {
        if (threadIdx.x == 0 && tile == 0) report_bad(A.err, 5, Rp, ra, rb, D);
        return;
    }
    const int i0 = (tile / A.tdim) * TS, j0 = (tile % A.tdim) * TS;
    if (i0 >= ra || j0 >= rb) return;
    const bool diag = P.ta == P.tb;
    if (diag && j0 > i0) return;                   // written by the mirror of tile (j0, i0)
    const bool mirror = diag && j0 < i0;
    const int dk = A.lay.dk;
    const uint16_t* wd = reinterpret_cast<const uint16_t*>(scr + A.lay.wd) + (size_t)P.ta * OZP * D * dk;
    const uint16_t* yd = reinterpret_cast<const uint16_t*>(scr + A.lay.yd) + (size_t)P.tb * OZP * D * dk;
    const int* we = reinterpret_cast<const int*>(scr + A.lay.we) + P.ta * D;
    const int* ye = reinterpret_cast<const int*>(scr + A.lay.ye) + P.tb * D;
    const int nr = min(TS, ra - i0), nc = min(TS, rb - j0);
    __shared__ __align__(16) uint16_t sA[OZP][TS][OZLD], sB[OZP][TS][OZLD];
    const int w = threadIdx.x / 32, l = threadIdx.x % 32, gid = l / 4, tig = l % 4;
    // warp tile: rows 16 mi .. 16 mi + 15, columns 8 ni .. 8 ni + 7
    const int mi = w / 4, ni = w % 4;
    const bool act = 16 * mi < nr && 8 * ni < nc;      // warp-uniform
    long long hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
    for (int k0 = 0; k0 < Rp; k0 += OZK) {
        const int kc = min(OZK, Rp - k0);
        // digit chunk: 2 operands x OZP digits x TS rows x 4 segments of 8 k
        for (int e = threadIdx.x; e < 2 * OZP * TS * 4; e += NT) {
            const int op = e / (OZP * TS * 4), p = (e / (TS * 4)) % OZP, r = (e / 4) % TS, c = e % 4;
            const int nrow = op ? nc : nr;
            const uint16_t* src = op ? yd : wd;
            const int row0 = op ? j0 : i0;
            int4 v = make_int4(0, 0, 0, 0);
            if (r < nrow) v = *reinterpret_cast<const int4*>(&src[((size_t)p * D + row0 + r) * dk + k0 + 8 * c]);
            *reinterpret_cast<int4*>(op ? &sB[p][r][8 * c] : &sA[p][r][8 * c]) = v;
        }
        __syncthreads();
        if (act) oz_warp_chunk(&sA[0][0][0], TS * OZLD, OZLD, &sB[0][0][0], TS * OZLD, OZLD, mi, ni, kc, hi, lo);
        __syncthreads();
    }
    double* B = slot_ptr(A.slots, P.slot, A.lanes, lane, D);
    double* sT = reinterpret_cast<double*>(&sA[0][0][0]);   // TS x (TS + 1), free after the k loop
    if (act) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int r = 16 * mi + gid + (c >= 2 ? 8 : 0), q = 8 * ni + 2 * tig + (c & 1);
            if (r < nr && q < nc) {
                const double v = oz_value(hi[c], lo[c], we[i0 + r], ye[j0 + q]);
                belem(B, D, P.trans, i0 + r, j0 + q) -= v;
                if (mirror) sT[r * (TS + 1) + q] = v;
            }
        }
    }
    if (mirror) {
        __syncthreads();
        schur_mirror(B, D, P.trans, i0, j0, nr, nc, sT, TS + 1, TS);
    }
}
__global__ void __launch_bounds__(NT, 3) k_schur_oz(SchurArgs A) { k_schur_oz_body(A, blockIdx.x, blockIdx.y); }
__global__ void __launch_bounds__(NT, 3) k_schur_oz_g(GroupArgs<SchurArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_schur_oz_body(G.args[m], blockIdx.x - G.off[m], blockIdx.y);
}

// ---- The same digit products on the 5th-generation tensor cores (tcgen05).
// Per (elimination, lane) the Schur updates of all target pairs form one
// block-lower-triangular product: the rows of W of every target stacked
// (target order, live rows only) against the rows of Y stacked the same way.
// One CTA takes a panel of 128 stacked rows of W: their 8 digit planes stay
// in shared memory (the MMA's A operand, M = 128), and the stacked rows of Y
// stream through in chunks of 32 (B operand, N = 32).  For every chunk one
// thread issues the 36 digit-pair products (K in steps of 16) into 8 FP32
// level accumulators in tensor memory (level s = p + q, 8 x 32 columns, two
// buffers).  A three-stage pipeline keeps the units busy: while the threads
// fold chunk c, the tensor core multiplies chunk c + 1 and cp.async brings
// chunk c + 2 into shared memory.  Warp w reads the tensor-memory lanes of its
// quarter (w mod 4: 32 panel rows) and folds 8 of the 32 columns (w / 4):
// every thread folds its row's 8 level sums of a column into the exact int64
// pair (hi, lo) of k_schur_oz and rounds once (oz_value).  With K <= 64 every
// level sum is an integer of magnitude < 8 * 64 * 127^2 < 2^23, exact in
// FP32.  The values, the element convention of diagonal pairs (32 x 32 tiles
// on the tile diagonal written whole, lower tiles also mirrored, upper tiles
// skipped) and hence the results are those of k_schur_oz.
// Operands sit in shared memory in the no-swizzle K-major layout of 8-row x
// 16-byte core matrices: element (r, k) of a plane at (r / 8) * 1024 +
// (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2 bytes (K-direction core stride
// 128 B, 8-row stride 1024 B).
constexpr int TCM = 128;                        // panel rows (MMA M)
constexpr int TCN = 32;                         // chunk rows of Y (MMA N)
constexpr int TCK = 64;                         // largest K held (digit columns)
constexpr int TC_THREADS = 512;                 // 16 warps: 4 per tensor-memory quarter
constexpr uint32_t TC_APLANE = TCM * TCK * 2;   // bytes of one digit plane of the panel
constexpr uint32_t TC_BPLANE = TCN * TCK * 2;   // bytes of one digit plane of a chunk
constexpr size_t TC_SMEM = (size_t)OZP * TC_APLANE + 2 * (size_t)OZP * TC_BPLANE;
constexpr long TC_WAIT_LIMIT = 1L << 26;        // polls of an mbarrier before giving up

__device__ __forceinline__ uint32_t tc_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, K-direction core stride
// (128 B), 8-row stride (1024 B), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, int accum) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
                 "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done = 0;
    for (long it = 0; it < TC_WAIT_LIMIT && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(tc_saddr(bar)), "r"(parity) : "memory");
    return done != 0;
}

// 16 bytes global -> shared without passing through registers; src_bytes = 0
// writes zeros (nothing is read)
__device__ __forceinline__ void tc_cp16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc_saddr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void tc_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void tc_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 8 consecutive TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// the stacked row g < pre[nt] as (target, row): targets are few, a linear scan
__device__ __forceinline__ int tc_target_of(const int* pre, int g) {
    int t = 0;
    while (pre[t + 1] <= g) ++t;
    return t;
}

__device__ __forceinline__ void k_schur_tc_body(const SchurArgs& A, const int bx, const int by) {
    HbScope hb_(5);
    const int lane = by;
    if (lane >= *A.active) return;
    const int ci = bx / A.npanel, panel = bx % A.npanel;
    const int D = A.D, dk = A.lay.dk;
    const double* scr = A.scratch + ((size_t)ci * A.lanes + lane) * A.lay.total;
    const int* hdr = (const int*)(scr + A.lay.hdr);
    const int Rp = hdr[1];
    const int nt = A.ntarg[ci];
    if (Rp <= 0 || nt <= 0) return;
    if (Rp > TCK || Rp > D || dk > TCK || nt > 64) {
        if (threadIdx.x == 0 && panel == 0) report_bad(A.err, 7, Rp, D, dk, nt);
        return;
    }
    // stacked live rows of the targets (prefix sums), the same for every thread
    __shared__ int pre[65];
    __shared__ int rowt[TCM], rowi[TCM];      // panel row -> (target, row)
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_poff;
    if (threadIdx.x == 0) {
        int acc = 0, bad = 0;
        pre[0] = 0;
        for (int t = 0; t < nt; ++t) {
            const int r = hdr[HDR_ROWS + t];
            bad |= (r < 0 || r > D);
            acc += max(0, min(r, D));
            pre[t + 1] = acc;
        }
        if (bad) report_bad(A.err, 7, Rp, D, nt, -1);
        int po = 0;                            // first pair of this elimination
        for (int c = 0; c < ci; ++c) po += A.ntarg[c] * (A.ntarg[c] + 1) / 2;
        s_poff = po;
    }
    __syncthreads();
    const int total = pre[nt];
    const int g0 = panel * TCM;
    if (g0 >= total) return;                   // uniform: nothing staged, nothing allocated
    if (threadIdx.x < TCM) {
        const int g = g0 + threadIdx.x;
        int t = -1, i = 0;
        if (g < total) {
            t = tc_target_of(pre, g);
            i = g - pre[t];
        }
        rowt[threadIdx.x] = t;
        rowi[threadIdx.x] = i;
    }
    __syncthreads();
    const int tmax = rowt[min(TCM, total - g0) - 1];
    const int colmax = pre[tmax + 1];          // pairs (t, u) need u <= t
    const int nchunk = (colmax + TCN - 1) / TCN;
    const int nks = (Rp + 15) / 16;            // K steps of 16 (zero digits up to 32-aligned Rp)
    const int nkc = 2 * nks;                   // 16-byte chunks of a staged row
    extern __shared__ __align__(128) uint8_t tcsm[];
    uint8_t* sA = tcsm;
    uint8_t* sB = tcsm + (size_t)OZP * TC_APLANE;
    const uint16_t* wd = reinterpret_cast<const uint16_t*>(scr + A.lay.wd);
    const uint16_t* yd = reinterpret_cast<const uint16_t*>(scr + A.lay.yd);
    const int* we = reinterpret_cast<const int*>(scr + A.lay.we);
    const int* ye = reinterpret_cast<const int*>(scr + A.lay.ye);
    // A: the panel's 8 digit planes (rows past the stack are zero)
    for (int e = threadIdx.x; e < OZP * TCM * nkc; e += TC_THREADS) {
        const int p = e / (TCM * nkc), rem = e % (TCM * nkc), r = rem / nkc, c = rem % nkc;
        const int t = rowt[r];
        const uint16_t* src = t >= 0 ? &wd[(((size_t)t * OZP + p) * D + rowi[r]) * dk + 8 * c] : wd;
        tc_cp16(sA + (size_t)p * TC_APLANE + (r / 8) * 1024 + c * 128 + (r % 8) * 16, src, t >= 0 ? 16 : 0);
    }
    tc_cp_commit();
    const int w = threadIdx.x / 32;
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_saddr(&tmem_base)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_saddr(&bar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_saddr(&bar[1])), "r"(1));
    }
    // cp.async of chunk c's 8 digit planes (stacked Y rows 32c ..) into buffer c % 2
    auto chunk_load = [&](int c) {
        uint8_t* dst = sB + (size_t)(c & 1) * OZP * TC_BPLANE;
        for (int e = threadIdx.x; e < OZP * TCN * nkc; e += TC_THREADS) {
            const int q = e / (TCN * nkc), rem = e % (TCN * nkc), r = rem / nkc, cc = rem % nkc;
            const int g = c * TCN + r;
            const uint16_t* src = yd;
            int nb = 0;
            if (g < colmax) {
                const int u = tc_target_of(pre, g);
                src = &yd[(((size_t)u * OZP + q) * D + (g - pre[u])) * dk + 8 * cc];
                nb = 16;
            }
            tc_cp16(dst + (size_t)q * TC_BPLANE + (r / 8) * 1024 + cc * 128 + (r % 8) * 16, src, nb);
        }
        tc_cp_commit();
    };
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TCN >> 3) << 17) | ((uint32_t)(TCM >> 4) << 24);
    // thread 0: the 36 x nks products of chunk c into tensor-memory buffer c % 2
    auto issue = [&](int c) {
        if (threadIdx.x != 0) return;
        const int b = c & 1;
        const uint32_t dcol = tmem_base + (uint32_t)(b * OZP * TCN);
        const uint32_t a0 = tc_saddr(sA), b0 = tc_saddr(sB + (size_t)b * OZP * TC_BPLANE);
        for (int lv = 0; lv < OZP; ++lv)
            for (int p = 0; p <= lv; ++p)
                for (int ks = 0; ks < nks; ++ks)
                    tc_mma(dcol + (uint32_t)(lv * TCN), tc_desc(a0 + p * TC_APLANE + ks * 256),
                           tc_desc(b0 + (lv - p) * TC_BPLANE + ks * 256), idesc, (p | ks) != 0);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         tc_saddr(&bar[b]))
                     : "memory");
    };
    // copies landed -> visible to the tensor core and to every thread; every
    // thread is done reading the tensor-memory buffer the next products reuse
    auto publish = [&]() {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    };
    // this thread's row (tensor-memory lane) and its 8 columns of every chunk
    const int quarter = w & 3, cgrp = w >> 2;
    const int R = 32 * quarter + (threadIdx.x & 31);
    const int myt = rowt[R], myi = rowi[R];
    const int myexp = myt >= 0 ? we[myt * D + myi] : 0;
    // prologue: A and chunk 0 landed, chunk 1 in flight, products of chunk 0
    chunk_load(0);
    if (nchunk > 1) {
        chunk_load(1);
        tc_cp_wait<1>();
    } else {
        tc_cp_wait<0>();
    }
    publish();
    issue(0);
    // Each thread waits for a chunk's products itself (bounded).  A wait that
    // runs out is reported and the loop goes on, so that every thread meets
    // the same barriers; the results of that call are then invalid.
    int timed_out = 0;
    for (int c = 0; c < nchunk; ++c) {
        const int b = c & 1;
        // this thread's 8 elements of chunk c: where they go, and S read early
        // (the loads overlap the wait for the products and the fold)
        const int gc = c * TCN + 8 * cgrp;         // this thread's first stacked column
        double* dst[8];
        double* mir[8];
        double s0[8];
        int ecol[8];
        {
            int u = gc < colmax ? tc_target_of(pre, gc) : nt;
            int j = gc < colmax ? gc - pre[u] : 0;
            double* Bk = nullptr;
            int trans = 0, ucur = -1;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                dst[jj] = nullptr;
                mir[jj] = nullptr;
                ecol[jj] = 0;
                const bool col_ok = gc + jj < colmax;
                if (col_ok && myt >= 0 && u <= myt && !(u == myt && myi / TS < j / TS)) {
                    if (u != ucur) {
                        const SchurPair P = A.pairs[s_poff + myt * (myt + 1) / 2 + u];
                        Bk = slot_ptr(A.slots, P.slot, A.lanes, lane, D);
                        trans = P.trans;
                        ucur = u;
                    }
                    dst[jj] = &belem(Bk, D, trans, myi, j);
                    if (u == myt && myi / TS > j / TS) mir[jj] = &belem(Bk, D, trans, j, myi);
                    ecol[jj] = ye[u * D + j];
                }
                if (col_ok && ++j == pre[u + 1] - pre[u]) {      // next stacked column
                    j = 0;
                    ++u;
                    while (u < nt - 1 && pre[u + 1] == pre[u]) ++u;
                }
            }
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) s0[jj] = dst[jj] ? *dst[jj] : 0.0;
        }
        if (!tc_wait(&bar[b], (uint32_t)((c >> 1) & 1))) timed_out = 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // chunk c + 2 into the buffer chunk c's products have released
        if (c + 2 < nchunk) chunk_load(c + 2);
        // chunk c + 1 landed: its products run while chunk c is folded
        if (c + 1 < nchunk) {
            if (c + 2 < nchunk) tc_cp_wait<1>();
            else tc_cp_wait<0>();
            publish();
            issue(c + 1);
        }
        const uint32_t taddr = tmem_base + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(b * OZP * TCN + 8 * cgrp);
        float lvv[OZP][8];
#pragma unroll
        for (int lv = 0; lv < OZP; ++lv) tc_ld8(taddr + (uint32_t)(lv * TCN), lvv[lv]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            if (!dst[jj]) continue;
            long long h = __float2int_rn(lvv[0][jj]);
            h = h * 128 + __float2int_rn(lvv[1][jj]);
            h = h * 128 + __float2int_rn(lvv[2][jj]);
            h = h * 128 + __float2int_rn(lvv[3][jj]);
            long long g = __float2int_rn(lvv[4][jj]);
            g = g * 128 + __float2int_rn(lvv[5][jj]);
            g = g * 128 + __float2int_rn(lvv[6][jj]);
            g = g * 128 + __float2int_rn(lvv[7][jj]);
            const double v = oz_value(h, g, myexp, ecol[jj]);
            *dst[jj] = s0[jj] - v;
            if (mir[jj]) *mir[jj] -= v;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (timed_out) report_bad(A.err, 7, nchunk, -2, -2, -2);
    tc_cp_wait<0>();
    __syncthreads();
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512));
}
__global__ void __launch_bounds__(TC_THREADS, 1) k_schur_tc(SchurArgs A) { k_schur_tc_body(A, blockIdx.x, blockIdx.y); }
__global__ void __launch_bounds__(TC_THREADS, 1) k_schur_tc_g(GroupArgs<SchurArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_schur_tc_body(G.args[m], blockIdx.x - G.off[m], blockIdx.y);
}

// Mixed path: S_ab[i0:i0+64, j0:j0+64] -= W_a Y_b^T (Eq. blr2-diag-schur) with
// FP32 products and accumulation; W, Y were stored in FP32 by k_trsm<float>.
// Thread (tx, ty) owns rows ty + 16 i and columns tx + 16 j (i, j < 4): the W
// reads are warp broadcasts, the Y reads hit 16 distinct banks, and the FP64
// read-modify-write of S is coalesced along rows.
__device__ __forceinline__ void k_schur_f32_body(const SchurArgs& A, const int bx, const int by) {
    HbScope hb_(5);
    const int lane = by;
    if (lane >= *A.active) return;
    const int pi = bx / A.tiles_per_pair, tile = bx % A.tiles_per_pair;
    const SchurPair P = A.pairs[pi];
    const int D = A.D;
    const double* scr = A.scratch + ((size_t)P.elim * A.lanes + lane) * A.lay.total;
    const int* hdr = (const int*)(scr + A.lay.hdr);
    const int Rp = hdr[1];
    if (Rp <= 0) return;
    const int ra = hdr[HDR_ROWS + P.ta], rb = hdr[HDR_ROWS + P.tb];
    if (Rp > D || ra < 0 || ra > D || rb < 0 || rb > D) {
        if (threadIdx.x == 0 && tile == 0) report_bad(A.err, 5, Rp, ra, rb, D);
        return;
    }
    const int i0 = (tile / A.tdim) * TSF, j0 = (tile % A.tdim) * TSF;
    if (i0 >= ra || j0 >= rb) return;
    const bool diag = P.ta == P.tb;
    if (diag && j0 > i0) return;                   // written by the mirror of tile (j0, i0)
    const bool mirror = diag && j0 < i0;
    const float* W = reinterpret_cast<const float*>(scr + A.lay.w + (size_t)P.ta * D * D);
    const float* Y = reinterpret_cast<const float*>(scr + A.lay.y + (size_t)P.tb * D * D);
    __shared__ float sbuf[2 * TSF * 33];            // the operand tiles, then the mirror's staging
    float(*sW)[33] = reinterpret_cast<float(*)[33]>(sbuf);
    float(*sY)[33] = reinterpret_cast<float(*)[33]>(sbuf + TSF * 33);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < Rp; k0 += 32) {
        const int kc = min(32, Rp - k0);
        for (int e = threadIdx.x; e < TSF * 32; e += NT) {
            int r = e / 32, k = e % 32;
            sW[r][k] = (i0 + r < ra && k < kc) ? W[(size_t)(i0 + r) * D + k0 + k] : 0.f;
            sY[r][k] = (j0 + r < rb && k < kc) ? Y[(size_t)(j0 + r) * D + k0 + k] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kc; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sW[ty + 16 * i][k];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sY[tx + 16 * j][k];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
    double* B = slot_ptr(A.slots, P.slot, A.lanes, lane, D);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int r = i0 + ty + 16 * i, c = j0 + tx + 16 * j;
            if (r < ra && c < rb) {
                belem(B, D, P.trans, r, c) -= (double)acc[i][j];
                if (mirror) sbuf[(ty + 16 * i) * (TSF + 1) + tx + 16 * j] = acc[i][j];
            }
        }
    if (mirror) {
        __syncthreads();
        schur_mirror(B, D, P.trans, i0, j0, min(TSF, ra - i0), min(TSF, rb - j0), sbuf, TSF + 1, TSF);
    }
}
__global__ void __launch_bounds__(NT) k_schur_f32(SchurArgs A) { k_schur_f32_body(A, blockIdx.x, blockIdx.y); }
__global__ void __launch_bounds__(NT) k_schur_f32_g(GroupArgs<SchurArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_schur_f32_body(G.args[m], blockIdx.x - G.off[m], blockIdx.y);
}

// leaf level: copy Q^T A Q near blocks, subtract sigma on the diagonal, fill
// blocks start as their coupling; dims/ranks from the build
struct InitArgs {
    double* slots;
    int D, lanes;
    const double* near_static;
    const int* slot_a;
    const int* slot_b;
    const int* slot_kind;
    const int* slot_far;
    const double* C;
    int rbl;
    const int* rb;
    const double* shifts;
    const int* active;
    double* stats;
};

__device__ __forceinline__ void k_init_leaf_body(const InitArgs& A, const int bx, const int by) {
    HbScope hb_(0);
    const int sl = bx, lane = by;
    if (lane >= *A.active) return;
    const int D = A.D;
    double* B = slot_ptr(A.slots, sl, A.lanes, lane, D);
    const int a = A.slot_a[sl], b = A.slot_b[sl];
    if (threadIdx.x == 0) atomicAdd(&A.stats[H2_NKINDS + H2_KIND_INIT], 16.0 * D * (double)D);
    if (A.slot_kind[sl] == 0) {
        const double* S = A.near_static + (size_t)sl * D * D;
        double sg = A.shifts[lane];
        for (int e = threadIdx.x; e < D * D; e += NT) {
            double v = S[e];
            if (a == b && (e / D) == (e % D)) v -= sg;
            B[e] = v;
        }
    } else {
        const double* C = A.C + (size_t)A.slot_far[sl] * A.rbl * A.rbl;
        int ra = A.rb[a], rbb = A.rb[b];
        for (int e = threadIdx.x; e < D * D; e += NT) {
            int i = e / D, j = e % D;
            B[e] = (i < ra && j < rbb) ? C[(size_t)i * A.rbl + j] : 0.0;
        }
    }
}
__global__ void k_init_leaf(InitArgs A) { k_init_leaf_body(A, blockIdx.x, blockIdx.y); }
__global__ void k_init_leaf_g(GroupArgs<InitArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_init_leaf_body(G.args[m], blockIdx.x - G.off[m], blockIdx.y);
}

__global__ void k_init_dims(int* dim, int* rk, const int64_t* off, const int* rb, int nc, int lanes,
                            unsigned long long* neg, unsigned long long* minpiv, int* err, double* stats) {
    HbScope hb_(8);
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nc * lanes) {
        int c = e / lanes;
        dim[e] = (int)(off[c + 1] - off[c]);
        rk[e] = rb[c];
    }
    if (e < lanes) {
        neg[e] = 0ull;
        minpiv[e] = (unsigned long long)__double_as_longlong(1.0 / 0.0);
    }
    (void)err;   // the error record persists until read (h2_status / host calls)
    if (e < 2 * H2_NKINDS) stats[e] = 0.0;
}

// parent dims: dim[P] = rk[c1] + rk[c2], rk[P] = rb[P]
__global__ void k_merge_dims(int* dimP, int* rkP, const int* rkC, const int* rbP, int ncP, int lanes) {
    HbScope hb_(9);
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ncP * lanes) return;
    int P = e / lanes, lane = e % lanes;
    dimP[e] = rkC[(2 * P) * lanes + lane] + rkC[(2 * P + 1) * lanes + lane];
    rkP[e] = rbP[P];
}

struct MergeArgs {
    double* slotsP;
    int DP, lanes;
    const int* slotP_a;
    const int* slotP_b;
    const int* slotP_kind;
    const int* slotP_far;
    const double* CP;
    int rblP;
    const int* rbP;
    const double* TP;
    int dqP;
    const double* slotsC;
    int DC;
    int ncC;
    const int* slot_ofC;
    const int* far_ofC;
    const double* CC;
    int rblC;
    const int* rbC;
    const int* rkC;
    double* scratch;   // [nslotsP][lanes][2][DP*DP]
    const int* active;
    double* stats;
    int* err;
};

__device__ __forceinline__ int place_child(int first, int i, int rb_self, int rb1, int rb2, int t1) {
    // parent coordinates [orig c1 | orig c2 | new c1 | new c2]
    if (i < rb_self) return first ? i : rb1 + i;
    return rb1 + rb2 + (first ? (i - rb_self) : t1 + (i - rb_self));
}

__device__ __forceinline__ void k_merge_body(const MergeArgs& A, const int bx, const int by) {
    HbScope hb_(6);
    const int sl = bx, lane = by;
    if (lane >= *A.active) return;
    const int DP = A.DP, LN = A.lanes;
    double* out = slot_ptr(A.slotsP, sl, LN, lane, DP);
    const int P = A.slotP_a[sl], Q = A.slotP_b[sl];
    if (A.slotP_kind[sl] == 1) {
        const double* C = A.CP + (size_t)A.slotP_far[sl] * A.rblP * A.rblP;
        int ra = A.rbP[P], rq = A.rbP[Q];
        for (int e = threadIdx.x; e < DP * DP; e += NT) {
            int i = e / DP, j = e % DP;
            out[e] = (i < ra && j < rq) ? C[(size_t)i * A.rblP + j] : 0.0;
        }
        return;
    }
    double* S = A.scratch + ((size_t)sl * LN + lane) * 2 * DP * DP;
    double* M = S + (size_t)DP * DP;
    int rkc[4], rbc[4];
    const int cc[4] = {2 * P, 2 * P + 1, 2 * Q, 2 * Q + 1};
    for (int u = 0; u < 4; ++u) {
        rkc[u] = A.rkC[cc[u] * LN + lane];
        rbc[u] = A.rbC[cc[u]];
    }
    const int dP = rkc[0] + rkc[1], dQ = rkc[2] + rkc[3];
    const int kP = rbc[0] + rbc[1], kQ = rbc[2] + rbc[3];
    {
        bool bad = dP > DP || dQ > DP || kP > A.dqP || kQ > A.dqP;
        for (int u = 0; u < 4; ++u) bad = bad || rkc[u] < rbc[u] || rkc[u] > A.DC;
        if (bad) {
            if (threadIdx.x == 0) report_bad(A.err, 6, dP, dQ, kP, kQ);
            return;
        }
    }
    if (threadIdx.x == 0) {
        atomicAdd(&A.stats[H2_KIND_MERGE], 2.0 * kP * (double)kP * dQ + 2.0 * dP * (double)kQ * kQ);
        atomicAdd(&A.stats[H2_NKINDS + H2_KIND_MERGE],
                  8.0 * (2.0 * dP * (double)dQ + (double)kP * kP + (double)kQ * kQ + (double)DP * DP));
    }
    for (int e = threadIdx.x; e < DP * DP; e += NT) S[e] = 0.0;
    __syncthreads();
    for (int u = 0; u < 2; ++u)
        for (int v = 2; v < 4; ++v) {
            const int c = cc[u], d = cc[v];
            const int rc_ = rkc[u], rd_ = rkc[v];
            const int sc = A.slot_ofC[(size_t)max(c, d) * A.ncC + min(c, d)];
            for (int e = threadIdx.x; e < rc_ * rd_; e += NT) {
                int i = e / rd_, j = e % rd_;
                double val;
                if (sc >= 0) {
                    const double* B = A.slotsC + ((size_t)sc * LN + lane) * (size_t)A.DC * A.DC;
                    val = c >= d ? B[(size_t)i * A.DC + j] : B[(size_t)j * A.DC + i];
                } else {
                    int fi = c > d ? A.far_ofC[(size_t)c * A.ncC + d] : A.far_ofC[(size_t)d * A.ncC + c];
                    const double* C = A.CC + (size_t)fi * A.rblC * A.rblC;
                    if (i < rbc[u] && j < rbc[v])
                        val = c > d ? C[(size_t)i * A.rblC + j] : C[(size_t)j * A.rblC + i];
                    else
                        val = 0.0;
                }
                int pi_ = place_child(u == 0, i, rbc[u], rbc[0], rbc[1], rkc[0] - rbc[0]);
                int pj_ = place_child(v == 2, j, rbc[v], rbc[2], rbc[3], rkc[2] - rbc[2]);
                S[(size_t)pi_ * DP + pj_] = val;
            }
        }
    __syncthreads();
    const double* TPm = A.TP + (size_t)P * A.dqP * A.dqP;
    const double* TQm = A.TP + (size_t)Q * A.dqP * A.dqP;
    for (int e = threadIdx.x; e < dP * dQ; e += NT) {     // M = T_P^T S
        int i = e / dQ, j = e % dQ;
        double v;
        if (i < kP) {
            v = 0.0;
            for (int k = 0; k < kP; ++k) v += TPm[(size_t)k * A.dqP + i] * S[(size_t)k * DP + j];
        } else {
            v = S[(size_t)i * DP + j];
        }
        M[(size_t)i * DP + j] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < DP * DP; e += NT) {     // out = M T_Q
        int i = e / DP, j = e % DP;
        double v = 0.0;
        if (i < dP && j < dQ) {
            if (j < kQ) {
                for (int k = 0; k < kQ; ++k) v += M[(size_t)i * DP + k] * TQm[(size_t)k * A.dqP + j];
            } else {
                v = M[(size_t)i * DP + j];
            }
        }
        out[e] = v;
    }
}
__global__ void __launch_bounds__(NT) k_merge(MergeArgs A) { k_merge_body(A, blockIdx.x, blockIdx.y); }
__global__ void __launch_bounds__(NT) k_merge_g(GroupArgs<MergeArgs> G) {
    const int m = group_find(G.off, G.n, blockIdx.x);
    k_merge_body(G.args[m], blockIdx.x - G.off[m], blockIdx.y);
}

__global__ void k_set_int(int* p, int v) {
    HbScope hb_(11);
    *p = v;
}

__global__ void k_finish(const unsigned long long* neg, const unsigned long long* minpiv, int64_t* counts,
                         double* mp, const int* active) {
    HbScope hb_(10);
    int lane = blockIdx.x * blockDim.x + threadIdx.x;
    if (lane >= *active) return;
    counts[lane] = (int64_t)neg[lane];
    mp[lane] = __longlong_as_double((long long)minpiv[lane]);
}

// ---- mixed-precision guard: certified counts (Parlett's criterion, Sec. 4.1)
// A mixed factorization of A~ - mu I is exact for A~ + E - mu I with ||E|| of
// the order of the FP32 product rounding.  Its count can differ from nu(mu)
// only if an eigenvalue lies within ||E|| of mu.  With Delta > 2 ||E||: if
// the mixed counts at mu - Delta and mu + Delta agree (= c), then nu is
// constant on [mu - Delta + ||E||, mu + Delta - ||E||], an interval around
// mu, so nu(mu) = c.  Shifts whose pair disagrees, or whose min |pivot| is
// below pivot_guard * ||A||_inf, are factorized again in FP64.

// lanes 2i and 2i + 1 of the next mixed batch: mu_i - Delta and mu_i + Delta
__global__ void k_guard_pairs(const double* req, int nc, double delta, double* shifts, int* active) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *active = 2 * nc;
    if (i < nc) {
        shifts[2 * i] = req[i] - delta;
        shifts[2 * i + 1] = req[i] + delta;
    }
}

// Certifies shifts c0 .. c0 + nc - 1 from the pair counts of the batch just
// run; the others are appended, in index order, to the FP64 list.  One CTA.
// tally[0] += shifts checked, tally[1] += shifts sent to FP64.
__global__ void __launch_bounds__(1024) k_guard_certify(const int64_t* cnt, const double* mp, int nc, int c0,
                                                        double theta, int64_t* out_c, double* out_mp,
                                                        int* rr_idx, int* rr_n, unsigned long long* tally) {
    __shared__ int wsum[32];
    __shared__ int s_base;
    const int t = threadIdx.x, w = t >> 5, l = t & 31, nw = (blockDim.x + 31) >> 5;
    if (t == 0) s_base = *rr_n;
    __syncthreads();
    for (int b0 = 0; b0 < nc; b0 += blockDim.x) {
        const int i = b0 + t;
        int f = 0;
        if (i < nc) {
            const int64_t a = cnt[2 * i], b = cnt[2 * i + 1];
            const double m = fmin(mp[2 * i], mp[2 * i + 1]);
            if (a == b && m >= theta) {
                out_c[c0 + i] = a;
                out_mp[c0 + i] = m;
            } else {
                f = 1;
            }
        }
        int incl = f;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (l >= o) incl += v;
        }
        if (l == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            int v = l < nw ? wsum[l] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if (l >= o) v += u;
            }
            if (l < nw) wsum[l] = v;
        }
        __syncthreads();
        if (f) rr_idx[s_base + (w > 0 ? wsum[w - 1] : 0) + incl - 1] = c0 + i;
        __syncthreads();
        if (t == 0) s_base += wsum[nw - 1];
        __syncthreads();
    }
    if (t == 0) {
        tally[1] += (unsigned long long)(s_base - *rr_n);
        tally[0] += (unsigned long long)nc;
        *rr_n = s_base;
    }
}

// a one-lane handle cannot hold a pair: every shift goes to FP64
__global__ void k_guard_all(int ns, int* rr_idx, int* rr_n, unsigned long long* tally) {
    for (int i = threadIdx.x; i < ns; i += blockDim.x) rr_idx[i] = i;
    if (threadIdx.x == 0) {
        *rr_n = ns;
        tally[0] += (unsigned long long)ns;
        tally[1] += (unsigned long long)ns;
    }
}

// the FP64 batch: shifts of the list in lanes 0 .. rr_n - 1
__global__ void k_guard_rerun_setup(const double* req, const int* rr_idx, const int* rr_n, double* shifts,
                                    int* active) {
    const int n = *rr_n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *active = n;
    if (i < n) shifts[i] = req[rr_idx[i]];
}

__global__ void k_guard_scatter(const int* rr_idx, const int* rr_n, const int64_t* cnt, const double* mp,
                                int64_t* out_c, double* out_mp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *rr_n) {
        out_c[rr_idx[i]] = cnt[i];
        out_mp[rr_idx[i]] = mp[i];
    }
}

// ------------------------------------------------------------ workspace --
constexpr size_t kSmemCap = 200 * 1024;   // dynamic shared memory staged per CTA at most
constexpr size_t kSmemMax = 227 * 1024;   // opt-in limit per CTA
// default Z width from which the recompression is shared by a cluster of QG CTAs
constexpr size_t kWideFill = 4096;

struct ColourDev {
    int ncl, ntarg_max, nrow_max, nfill_max, npairs, has_fill;
    int *cl, *targ, *targ_slot, *targ_trans, *ntarg, *rowblk, *rowblk_other, *rowblk_trans, *rowblk_fill,
        *nrow, *fillq, *fillslot, *nfill;
    SchurPair* pairs;
    // lookahead schedule: the pairs whose block lies in a row or column of a
    // cluster of the next colour (A), and the rest (B), in their list order
    SchurPair *pairsA, *pairsB;
    int npairsA, npairsB;
};

struct LevelWork {
    std::vector<ColourDev> colours;
    ScratchLayout lay;
    int ncl_max = 0;
    int* d_slot_of = nullptr;
    int* d_far_of = nullptr;
};

// Parameters of the device-resident bisection loop (set before each launch of
// its graph): the brackets in use and the width to reach; round statistics.
struct KthLoop {
    int nk;
    double width;
    int max_rounds;
    int rounds;                 // rounds with work in this launch
    unsigned long long shifts;  // shifts evaluated in this launch
    int stopped;                // 1: the round cap ended the loop
    int per_interval;           // shifts per interval and round (0: all lanes)
};

struct FactorState {
    std::vector<LevelWork> lw;
    int* d_active = nullptr;
    int64_t* d_counts = nullptr;
    double* d_mp = nullptr;
    double* d_stats = nullptr;  // [2 * H2_NKINDS]
    double* d_lo = nullptr;   // bisection
    double* d_hi = nullptr;
    int64_t* d_k = nullptr;
    int* d_nact = nullptr;
    int* d_first = nullptr;   // [lanes]: the intervals of a round
    int nk_cap = 0;
    // mixed-precision guard: requested shifts, certified results, FP64 list
    double* d_req = nullptr;      // [lanes]
    int64_t* d_gc = nullptr;      // [lanes]
    double* d_gmp = nullptr;      // [lanes]
    int* d_rr_idx = nullptr;      // [lanes]
    int* d_rr_n = nullptr;        // [1]
    unsigned long long* d_tally = nullptr;   // [2]: shifts checked, shifts re-run in FP64
    // lookahead schedule: the second stream of the fork and its two events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // device-resident bisection loop (graph with a conditional WHILE node)
    KthLoop* d_loop = nullptr;
    cudaGraphExec_t loop_exec[2] = {nullptr, nullptr};   // [mixed]
    int loop_nk_cap = 0;          // bracket capacity the loop graphs were built for
};

static FactorState* state_of(h2_matrix* h) {
    return reinterpret_cast<FactorState*>(h->ws.graph_state);
}

static int ensure_graph(h2_matrix* h, int mixed);
static int autotune(h2_matrix* h);
static void guard_pairs(h2_matrix* h, int c0, int nc);
static void guard_certify(h2_matrix* h, int c0, int nc);
static void guard_rerun_setup(h2_matrix* h);
static void guard_scatter(h2_matrix* h);
// graphs unless the handle asks for plain launches or the environment
// variable H2_NO_GRAPH=1 (a diagnostic) turns them off for the process
static bool use_graphs(const h2_matrix* h) {
    static const int no_graph = [] {
        const char* e = getenv("H2_NO_GRAPH");
        return e && e[0] == '1';
    }();
    return !no_graph && h->opt.graphs != 0;
}
int heartbeat_setup();

// the lookahead schedule (h2_options.lookahead) applies to a handle's own
// graph-replayed batches
static bool lookahead_on(const h2_matrix* h) { return h->opt.lookahead != 0 && use_graphs(h); }

// padded block dimension of every level (leaves: the largest leaf; above:
// twice the children's skeleton cap)
static int set_level_dims(h2_matrix* h) {
    const int L = h->plan.L;
    const int fill_cap = h->opt.fill_cap > 0 ? h->opt.fill_cap : 2 * h->rank;
    h->fill_cap_eff = fill_cap;
    for (int l = L; l >= 0; --l) {
        LevelDev& D = h->lev[l];
        if (l == L) D.dmax = std::max(1, h->mmax);
        else {
            const LevelDev& C = h->lev[l + 1];
            int skc = std::max(C.rbmax, std::min(fill_cap, C.dmax));
            D.dmax = std::max(1, 2 * skc);
        }
        if (rotate_smem<float>(D.dmax) > kSmemMax || (size_t)D.dmax * RC * sizeof(double) > kSmemMax) {
            set_error("block dimension " + std::to_string(D.dmax) + " exceeds the shared-memory staging of the rotation kernel");
            return H2_ERR_INVALID_ARG;
        }
    }
    return H2_OK;
}

// largest near count, near-or-fill count and fill count of a cluster of level l
static void level_maxima(const LevelPlan& lp, int* ntarg_max, int* nrow_max, int* nfill_max) {
    *ntarg_max = *nrow_max = *nfill_max = 1;
    for (int p = 0; p < lp.nc; ++p) {
        int nn = 0, nf = 0;
        for (int x = 0; x < lp.nc; ++x) {
            nn += lp.is_near(p, x);
            nf += lp.is_fill(p, x);
        }
        *ntarg_max = std::max(*ntarg_max, nn);
        *nrow_max = std::max(*nrow_max, nn + nf);
        *nfill_max = std::max(*nfill_max, nf);
    }
}

// Device bytes of the workspace per lane (every buffer of alloc_workspace
// grows linearly with the lanes; the work lists do not depend on them).
size_t workspace_lane_bytes(h2_matrix* h) {
    if (set_level_dims(h)) return 0;
    const Plan& P = h->plan;
    size_t slots = 0, scratch = 0, merge = 0;
    for (int l = 0; l <= P.L; ++l) {
        const LevelDev& D = h->lev[l];
        const LevelPlan& lp = P.lev[l];
        int nt, nr, nf;
        level_maxima(lp, &nt, &nr, &nf);
        const ScratchLayout lay = scratch_layout(D.dmax, nf, nt, h->opt.precision == H2_PREC_FP64_TC);
        size_t ncl_max = 0;
        for (const auto& cl : lp.color_lists) ncl_max = std::max(ncl_max, cl.size());
        slots += (size_t)std::max(D.nslots, 1) * D.dmax * D.dmax * 8 + (size_t)D.nc * 8;
        scratch = std::max(scratch, ncl_max * lay.total * 8 * (lookahead_on(h) ? 2 : 1));
        if (l < P.L) merge = std::max(merge, (size_t)D.nslots * 2 * D.dmax * D.dmax * 8);
    }
    return slots + scratch + merge + 5 * 8;
}

int alloc_workspace(h2_matrix* h, int lanes) {
    int hrc = heartbeat_setup();
    if (hrc) return hrc;
    const Plan& P = h->plan;
    const int L = P.L;
    Workspace& ws = h->ws;
    ws.lanes = lanes;
    auto* fs = new FactorState();
    ws.graph_state = fs;
    fs->lw.resize(L + 1);
    if ((hrc = set_level_dims(h))) return hrc;
    {   // admission by footprint: fail before allocating when the workspace cannot fit
        const size_t need = workspace_lane_bytes(h) * (size_t)lanes;
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        if (need > free_b) {
            set_error("workspace of " + std::to_string(lanes) + " lanes needs " + std::to_string(need) +
                      " bytes, " + std::to_string(free_b) + " free on the device");
            return H2_ERR_OOM;
        }
    }
    size_t scratch_max = 0, merge_max = 0;
    int rc;
    for (int l = 0; l <= L; ++l) {
        LevelDev& D = h->lev[l];
        const LevelPlan& lp = P.lev[l];
        LevelWork& W = fs->lw[l];
        int nc = lp.nc;
        int ntarg_max, nrow_max, nfill_max;
        level_maxima(lp, &ntarg_max, &nrow_max, &nfill_max);
        W.lay = scratch_layout(D.dmax, nfill_max, ntarg_max, h->opt.precision == H2_PREC_FP64_TC);
        for (const auto& cl : lp.color_lists) W.ncl_max = std::max<int>(W.ncl_max, (int)cl.size());
        scratch_max = std::max(scratch_max, (size_t)W.ncl_max * lanes * W.lay.total);
        if (l < L) merge_max = std::max(merge_max, (size_t)D.nslots * lanes * 2 * D.dmax * D.dmax);
        // colour work lists
        for (const auto& cl : lp.color_lists) {
            ColourDev C{};
            C.has_fill = 0;
            C.ncl = (int)cl.size();
            C.ntarg_max = ntarg_max;
            C.nrow_max = nrow_max;
            C.nfill_max = nfill_max;
            std::vector<int> targ(C.ncl * ntarg_max, -1), tslot(C.ncl * ntarg_max, -1),
                ttr(C.ncl * ntarg_max, 0), ntarg(C.ncl), rowblk(C.ncl * nrow_max, -1),
                rowother(C.ncl * nrow_max, -1), rowtr(C.ncl * nrow_max, 0), rowfill(C.ncl * nrow_max, 0),
                nrow(C.ncl),
                fillq(C.ncl * nfill_max, -1), fillslot(C.ncl * nfill_max, -1), nfill(C.ncl);
            std::vector<SchurPair> pairs;
            auto slot = [&](int a, int b) { return D.slot_of[(size_t)std::max(a, b) * nc + std::min(a, b)]; };
            for (int ci = 0; ci < C.ncl; ++ci) {
                int p = cl[ci];
                std::vector<int> tg{p};
                for (int x = 0; x < nc; ++x)
                    if (x != p && lp.is_near(p, x)) tg.push_back(x);
                ntarg[ci] = (int)tg.size();
                for (int ti = 0; ti < (int)tg.size(); ++ti) {
                    int a = tg[ti];
                    targ[ci * ntarg_max + ti] = a;
                    tslot[ci * ntarg_max + ti] = slot(a, p);
                    ttr[ci * ntarg_max + ti] = p > a ? 1 : 0;
                }
                for (int i = 0; i < (int)tg.size(); ++i)
                    for (int j = 0; j <= i; ++j) {
                        int a = tg[i], b = tg[j];
                        pairs.push_back(SchurPair{ci, i, j, slot(a, b), a < b ? 1 : 0, a, b});
                    }
                int nr = 0, nfl = 0;
                for (int x = 0; x < nc; ++x) {
                    if (lp.is_near(p, x) || lp.is_fill(p, x)) {
                        rowblk[ci * nrow_max + nr] = slot(p, x);
                        rowother[ci * nrow_max + nr] = x;
                        rowtr[ci * nrow_max + nr] = x > p ? 1 : 0;
                        rowfill[ci * nrow_max + nr] = lp.is_fill(p, x) ? 1 : 0;
                        ++nr;
                    }
                    if (lp.is_fill(p, x)) {
                        fillq[ci * nfill_max + nfl] = x;
                        fillslot[ci * nfill_max + nfl] = slot(p, x);
                        ++nfl;
                    }
                }
                nrow[ci] = nr;
                nfill[ci] = nfl;
                if (nfl > 0) C.has_fill = 1;
            }
            C.npairs = (int)pairs.size();
            {
                const size_t ci_now = W.colours.size();
                std::vector<char> in_next(nc, 0);
                if (ci_now + 1 < lp.color_lists.size())
                    for (int q : lp.color_lists[ci_now + 1]) in_next[q] = 1;
                std::vector<SchurPair> pa, pb;
                for (const SchurPair& sp : pairs) (in_next[sp.a] || in_next[sp.b] ? pa : pb).push_back(sp);
                C.npairsA = (int)pa.size();
                C.npairsB = (int)pb.size();
                if ((rc = upload(&C.pairsA, pa)) || (rc = upload(&C.pairsB, pb))) return rc;
            }
            if ((rc = upload(&C.cl, std::vector<int>(cl.begin(), cl.end()))) || (rc = upload(&C.targ, targ)) ||
                (rc = upload(&C.targ_slot, tslot)) || (rc = upload(&C.targ_trans, ttr)) ||
                (rc = upload(&C.ntarg, ntarg)) || (rc = upload(&C.rowblk, rowblk)) ||
                (rc = upload(&C.rowblk_other, rowother)) || (rc = upload(&C.rowblk_trans, rowtr)) ||
                (rc = upload(&C.rowblk_fill, rowfill)) ||
                (rc = upload(&C.nrow, nrow)) || (rc = upload(&C.fillq, fillq)) ||
                (rc = upload(&C.fillslot, fillslot)) || (rc = upload(&C.nfill, nfill)) ||
                (rc = upload(&C.pairs, pairs)))
                return rc;
            W.colours.push_back(C);
        }
        if ((rc = upload(&W.d_slot_of, D.slot_of)) || (rc = upload(&W.d_far_of, D.far_of))) return rc;
    }
    CK(cudaFuncSetAttribute(k_rotate_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    CK(cudaFuncSetAttribute(k_rotate_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    CK(cudaFuncSetAttribute(k_rotate<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    CK(cudaFuncSetAttribute(k_rotate<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    CK(cudaFuncSetAttribute(k_rotate<float, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    CK(cudaFuncSetAttribute(k_ldl<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap + 8192));
    CK(cudaFuncSetAttribute(k_ldl<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap + 8192));
    CK(cudaFuncSetAttribute(k_ldl_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    CK(cudaFuncSetAttribute(k_trsm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap + 8192));
    CK(cudaFuncSetAttribute(k_trsm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap + 8192));
    CK(cudaFuncSetAttribute(k_schur_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    // buffers
    ws.d_slots.assign(L + 1, nullptr);
    ws.d_dim.assign(L + 1, nullptr);
    ws.d_rk.assign(L + 1, nullptr);
    size_t bytes = 0;
    for (int l = 0; l <= L; ++l) {
        LevelDev& D = h->lev[l];
        size_t sz = (size_t)std::max(D.nslots, 1) * lanes * D.dmax * D.dmax;
        if ((rc = dalloc(&ws.d_slots[l], sz))) return rc;
        if ((rc = dalloc(&ws.d_dim[l], (size_t)D.nc * lanes))) return rc;
        if ((rc = dalloc(&ws.d_rk[l], (size_t)D.nc * lanes))) return rc;
        bytes += sz * 8 + (size_t)D.nc * lanes * 8;
    }
    // the lookahead schedule runs colour c + 1's solves while colour c's Schur
    // updates read their factors: two scratch halves, by colour parity
    ws.scratch_half = scratch_max;
    if ((rc = dalloc(&ws.d_scratch, (lookahead_on(h) ? 2 : 1) * scratch_max))) return rc;
    if (lookahead_on(h)) {
        CK(cudaStreamCreateWithFlags(&fs->side, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&fs->ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&fs->ev_join, cudaEventDisableTiming));
    }
    if ((rc = dalloc(&ws.d_merge, std::max<size_t>(merge_max, 1)))) return rc;
    bytes += ((lookahead_on(h) ? 2 : 1) * scratch_max + merge_max) * 8;
    if ((rc = dalloc(&ws.d_neg, lanes)) || (rc = dalloc(&ws.d_minpiv, lanes)) || (rc = dalloc(&ws.d_err, 8)) ||
        (rc = dalloc(&ws.d_shifts, lanes)) || (rc = dalloc(&fs->d_active, 1)) ||
        (rc = dalloc(&fs->d_counts, lanes)) || (rc = dalloc(&fs->d_mp, lanes)) ||
        (rc = dalloc(&fs->d_stats, 2 * H2_NKINDS)) || (rc = dalloc(&fs->d_req, lanes)) ||
        (rc = dalloc(&fs->d_gc, lanes)) || (rc = dalloc(&fs->d_gmp, lanes)) || (rc = dalloc(&fs->d_rr_idx, lanes)) ||
        (rc = dalloc(&fs->d_rr_n, 1)) || (rc = dalloc(&fs->d_tally, 2)))
        return rc;
    CK(cudaMemsetAsync(fs->d_tally, 0, 2 * sizeof(unsigned long long), h->stream));
    ws.bytes = bytes;
    CK(cudaMemsetAsync(ws.d_err, 0, 8 * sizeof(int), h->stream));
    // capture the batch graphs now, while nothing else runs on the device:
    // a capture never overlaps other handles' work on other streams
    CK(cudaStreamSynchronize(h->stream));
    if (h->opt.autotune && (rc = autotune(h))) return rc;
    if (use_graphs(h)) {
        if ((rc = ensure_graph(h, 0))) return rc;
        if (h->opt.precision == H2_PREC_MIXED && (rc = ensure_graph(h, 1))) return rc;
    }
    CK(cudaStreamSynchronize(h->stream));
    return H2_OK;
}

// Event pairs around launches (profiling mode of enqueue_factorization).
struct Profiler {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    size_t used = 0;
    cudaStream_t st = nullptr;
    void before(int k) {
        if (used + 2 > ev.size()) {
            for (int i = 0; i < 64; ++i) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                ev.push_back(e);
            }
        }
        kind.push_back(k);
        cudaEventRecord(ev[used++], st);
    }
    void after() { cudaEventRecord(ev[used++], st); }
};

// One launch of a batch, described before it is launched, so that a single
// handle launches its records one by one and a group of handles merges the
// records of equal key (step, colour, operation, variant) into one grouped
// launch (h2_group).  The 1-D bookkeeping kernels are kept as closures.
enum Op {
    OP_INIT_DIMS, OP_INIT_LEAF, OP_RECOMP, OP_RECOMP_CL, OP_ROTATE, OP_LDL, OP_TRSM, OP_SCHUR,
    OP_MERGE_DIMS, OP_MERGE, OP_FINISH, OP_FORK, OP_JOIN
};

struct LaunchRec {
    int op = 0, kind = 0;
    int phase = 0, step = 0, colour = 0;   // order key across handles
    int variant = 0;                       // template choice (see launch_single)
    dim3 grid;
    int block = NT;
    size_t smem = 0;
    int flag = 0;
    int branch = 0;                        // lookahead schedule: 1 = the side stream
    FactorArgs fa{};
    SchurArgs sa{};
    InitArgs ia{};
    MergeArgs ma{};
    std::function<void(cudaStream_t)> tiny;
};

// kernel choices of a level: autotuned when the handle has them, else the
// fixed rules (128 threads for blocks up to 64, clusters for wide Z)
static int ldl_threads(const h2_matrix* h, int l, int Dm) {
    if (l < (int)h->tune_ldl.size() && h->tune_ldl[l] > 0) return (h->tune_ldl[l] == 32 && Dm > 64) ? NT : h->tune_ldl[l];
    return Dm <= 64 ? 128 : NT;
}
static bool recomp_clustered(const h2_matrix* h, int l, int nfill_max, int Dm) {
    if (l < (int)h->tune_recomp.size() && h->tune_recomp[l] >= 0) return h->tune_recomp[l] == 1;
    const int wide = h->opt.recomp_cluster_cols;
    return wide >= 0 && (size_t)nfill_max * Dm >= (wide > 0 ? (size_t)wide : kWideFill);
}

static std::vector<LaunchRec> factor_records(h2_matrix* h, int mixed, bool lookahead = false) {
    std::vector<LaunchRec> R;
    const Plan& P = h->plan;
    const int L = P.L;
    Workspace& ws = h->ws;
    FactorState* fs = state_of(h);
    const int LN = ws.lanes;
    {
        LevelDev& D = h->lev[L];
        const int ne = std::max(std::max(D.nc * LN, LN), 2 * H2_NKINDS);
        LaunchRec r;
        r.op = OP_INIT_DIMS;
        r.kind = H2_KIND_OTHER;
        r.phase = 0;
        int* dim = ws.d_dim[L];
        int* rk = ws.d_rk[L];
        const int64_t* off = D.d_off;
        const int* rb = D.d_rb;
        const int nc = D.nc;
        unsigned long long* neg = ws.d_neg;
        unsigned long long* mp = ws.d_minpiv;
        int* err = ws.d_err;
        double* stats = fs->d_stats;
        r.tiny = [=](cudaStream_t st) {
            k_init_dims<<<(ne + 255) / 256, 256, 0, st>>>(dim, rk, off, rb, nc, LN, neg, mp, err, stats);
        };
        R.push_back(r);
        LaunchRec q;
        q.op = OP_INIT_LEAF;
        q.kind = H2_KIND_INIT;
        q.phase = 1;
        q.ia = InitArgs{ws.d_slots[L], D.dmax, LN, D.d_near_static, D.d_slot_a, D.d_slot_b, D.d_slot_kind,
                        D.d_slot_far, D.d_C, D.estride, D.d_rb, ws.d_shifts, fs->d_active, fs->d_stats};
        q.grid = dim3(D.nslots, LN);
        R.push_back(q);
    }
    for (int l = L; l >= 0; --l) {
        LevelDev& D = h->lev[l];
        LevelWork& W = fs->lw[l];
        const int Dm = D.dmax;
        const int ncol = (int)W.colours.size();
        // the records of colour c: its chain (recompression, rotation, LDL^T,
        // solves) and its Schur update, whole and split into the pairs in rows
        // and columns of the next colour's clusters (A) and the others (B)
        struct ColourRecs {
            std::vector<LaunchRec> chain;
            LaunchRec schur, schurA, schurB;
        };
        auto colour_recs = [&](int c) {
            ColourRecs out;
            const ColourDev& C = W.colours[c];
            double* scr = ws.d_scratch + ((lookahead && (c & 1)) ? ws.scratch_half : 0);
            FactorArgs fa{ws.d_slots[l], D.dmax, LN, ws.d_dim[l], ws.d_rk[l], D.d_color, c, C.cl, C.targ,
                          C.targ_slot, C.targ_trans, C.ntarg, C.ntarg_max, C.rowblk, C.rowblk_other,
                          C.rowblk_trans, C.rowblk_fill, C.nrow, C.nrow_max, C.fillq, C.fillslot, C.nfill,
                          C.nfill_max, scr, W.lay, h->tol, 2.220446049250313e-16 * h->norm_inf,
                          h->fill_cap_eff, ws.d_neg, ws.d_minpiv, ws.d_err, fs->d_active, fs->d_stats, C.ncl};
            LaunchRec r;
            r.phase = 2;
            r.step = L - l;
            r.colour = c;
            r.fa = fa;
            if (C.has_fill) {
                LaunchRec q = r;
                q.kind = H2_KIND_RECOMP;
                if (recomp_clustered(h, l, C.nfill_max, Dm)) {
                    q.op = OP_RECOMP_CL;
                    q.grid = dim3(C.ncl * QG, LN);
                    q.smem = (size_t)Dm * sizeof(double);
                } else {
                    q.op = OP_RECOMP;
                    q.grid = dim3(C.ncl, LN);
                }
                out.chain.push_back(q);
                q = r;
                q.op = OP_ROTATE;
                q.kind = H2_KIND_ROTATE;
                q.grid = dim3(C.ncl * C.nrow_max, LN);
                if (!mixed && h->opt.precision == H2_PREC_FP64_TC && rotate_oz_smem(Dm) <= kSmemMax) {
                    q.variant = 2;
                    q.smem = rotate_oz_smem(Dm);
                } else if (!mixed) {
                    q.variant = 0;
                    q.smem = (size_t)Dm * RC * sizeof(double);
                } else {
                    q.variant = rotate_nu(Dm);
                    q.smem = rotate_smem<float>(Dm);
                }
                out.chain.push_back(q);
            }
            {
                const size_t sm_ldl = ((size_t)Dm * (Dm + 1) + 4 * (size_t)Dm) * sizeof(double);
                LaunchRec q = r;
                q.op = OP_LDL;
                q.kind = H2_KIND_LDL;
                q.flag = sm_ldl <= kSmemCap ? 1 : 0;
                q.variant = ldl_threads(h, l, Dm);
                if (q.variant == 32) {           // one warp per block
                    q.block = 32 * LW;
                    q.flag = 1;
                    q.smem = LW * ldl_warp_slice(Dm) * sizeof(double);
                    q.grid = dim3((C.ncl * LN + LW - 1) / LW, 1);
                } else {
                    q.block = q.variant;
                    q.smem = q.flag ? sm_ldl : 0;
                    q.grid = dim3(C.ncl, LN);
                }
                out.chain.push_back(q);
            }
            {
                // flags 0 and 1: Rp pivot reciprocals, then (flag 1) L and the pivots
                const size_t sm_rc = (size_t)Dm * sizeof(double);
                const size_t sm_trsm = sm_rc + (size_t)Dm * (Dm + 1) * sizeof(double) + 2 * (size_t)Dm * sizeof(int);
                // flag 2: L, D and W staged (Rp (Rp + 1) + rows (Rp + 1) + 3 Rp values, 2 Rp ints)
                const size_t sm_full = ((size_t)Dm * (Dm + 1) + (size_t)Dm * (Dm + 1) + 3 * (size_t)Dm) * sizeof(double) +
                                       2 * (size_t)Dm * sizeof(int);
                LaunchRec q = r;
                q.op = OP_TRSM;
                q.kind = H2_KIND_TRSM;
                q.flag = sm_full <= kSmemCap ? 2 : (sm_trsm <= kSmemCap ? 1 : 0);
                q.variant = mixed ? 1 : 0;
                q.smem = q.flag == 2 ? sm_full : (q.flag ? sm_trsm : sm_rc);
                q.grid = dim3(C.ncl * C.ntarg_max, LN);
                out.chain.push_back(q);
            }
            {
                const int ts = mixed ? TSF : TS;
                const int tdim = (D.dmax + ts - 1) / ts;
                const int npanel = (C.ntarg_max * D.dmax + TCM - 1) / TCM;
                LaunchRec q = r;
                q.op = OP_SCHUR;
                q.kind = H2_KIND_SCHUR;
                q.sa = SchurArgs{ws.d_slots[l], D.dmax, LN, C.pairs, tdim * tdim, tdim, scr, W.lay,
                                 fs->d_active, ws.d_err, C.ntarg, npanel};
                q.variant = mixed ? 1 : (h->opt.precision == H2_PREC_FP64_TC ? 2 : 0);
                q.grid = dim3(C.npairs * tdim * tdim, LN);
                // FP64_TC with blocks of at most 64 rows: the tcgen05 kernel (one
                // CTA per 128-row panel of an elimination's stacked targets)
                if (q.variant == 2 && h->opt.tc_schur != 0 && D.dmax <= TCK && W.lay.dk <= TCK) {
                    q.variant = 3;
                    q.block = TC_THREADS;
                    q.smem = TC_SMEM;
                    q.grid = dim3(C.ncl * npanel, LN);
                }
                out.schur = q;
                out.schurA = q;
                out.schurA.sa.pairs = C.pairsA;
                out.schurA.grid = dim3(C.npairsA * tdim * tdim, LN);
                out.schurB = q;
                out.schurB.sa.pairs = C.pairsB;
                out.schurB.grid = dim3(C.npairsB * tdim * tdim, LN);
                out.schurB.branch = 1;
            }
            return out;
        };
        if (!lookahead) {
            for (int c = 0; c < ncol; ++c) {
                ColourRecs cr = colour_recs(c);
                for (auto& q : cr.chain) R.push_back(q);
                R.push_back(cr.schur);
            }
        } else {
            // the lookahead schedule: after colour c's Schur updates in the next
            // colour's rows and columns, colour c + 1's chain runs on the main
            // stream while the rest of colour c's Schur updates run on the side
            // stream; every block still takes its updates in the same order
            std::vector<ColourRecs> crs;
            for (int c = 0; c < ncol; ++c) crs.push_back(colour_recs(c));
            for (auto& q : crs[0].chain) R.push_back(q);
            for (int c = 0; c < ncol; ++c) {
                const bool split = c + 1 < ncol && crs[c].schur.variant != 3;
                if (!split) {
                    R.push_back(crs[c].schur);
                    if (c + 1 < ncol)
                        for (auto& q : crs[c + 1].chain) R.push_back(q);
                    continue;
                }
                if (crs[c].schurA.grid.x > 0) R.push_back(crs[c].schurA);
                LaunchRec fk;
                fk.op = OP_FORK;
                R.push_back(fk);
                if (crs[c].schurB.grid.x > 0) R.push_back(crs[c].schurB);
                for (auto& q : crs[c + 1].chain) R.push_back(q);
                LaunchRec jn;
                jn.op = OP_JOIN;
                R.push_back(jn);
            }
        }
        if (l > 0) {
            LevelDev& Pd = h->lev[l - 1];
            LaunchRec q;
            q.phase = 2;
            q.step = L - l;
            q.colour = 1 << 20;          // after every colour of the step
            q.op = OP_MERGE_DIMS;
            q.kind = H2_KIND_OTHER;
            const int ne = Pd.nc * LN;
            int* dimP = ws.d_dim[l - 1];
            int* rkP = ws.d_rk[l - 1];
            const int* rkC = ws.d_rk[l];
            const int* rbP = Pd.d_rb;
            const int ncP = Pd.nc;
            q.tiny = [=](cudaStream_t st) {
                k_merge_dims<<<(ne + 255) / 256, 256, 0, st>>>(dimP, rkP, rkC, rbP, ncP, LN);
            };
            R.push_back(q);
            LaunchRec m;
            m.phase = 2;
            m.step = L - l;
            m.colour = 1 << 20;
            m.op = OP_MERGE;
            m.kind = H2_KIND_MERGE;
            m.ma = MergeArgs{ws.d_slots[l - 1], Pd.dmax, LN, Pd.d_slot_a, Pd.d_slot_b, Pd.d_slot_kind,
                             Pd.d_slot_far, Pd.d_C, Pd.estride, Pd.d_rb, Pd.d_Q, Pd.dq, ws.d_slots[l], D.dmax,
                             D.nc, W.d_slot_of, W.d_far_of, D.d_C, D.estride, D.d_rb, ws.d_rk[l], ws.d_merge,
                             fs->d_active, fs->d_stats, ws.d_err};
            m.grid = dim3(Pd.nslots, LN);
            R.push_back(m);
        }
    }
    LaunchRec f;
    f.phase = 3;
    f.op = OP_FINISH;
    f.kind = H2_KIND_OTHER;
    unsigned long long* neg = ws.d_neg;
    unsigned long long* mp = ws.d_minpiv;
    int64_t* counts = fs->d_counts;
    double* dmp = fs->d_mp;
    int* act = fs->d_active;
    f.tiny = [=](cudaStream_t st) { k_finish<<<(LN + 255) / 256, 256, 0, st>>>(neg, mp, counts, dmp, act); };
    R.push_back(f);
    return R;
}

static void launch_single(const LaunchRec& r, cudaStream_t st) {
    switch (r.op) {
        case OP_INIT_LEAF: k_init_leaf<<<r.grid, NT, 0, st>>>(r.ia); break;
        case OP_RECOMP: k_recomp<<<r.grid, NT, 0, st>>>(r.fa); break;
        case OP_RECOMP_CL: k_recomp_cluster<<<r.grid, NT, r.smem, st>>>(r.fa); break;
        case OP_ROTATE:
            if (r.variant == 0) k_rotate_fp64<<<r.grid, NT, r.smem, st>>>(r.fa);
            else if (r.variant == 2) k_rotate_oz<<<r.grid, NT, r.smem, st>>>(r.fa);
            else if (r.variant == 8) k_rotate<float, 8><<<r.grid, NT, r.smem, st>>>(r.fa);
            else if (r.variant == 16) k_rotate<float, 16><<<r.grid, NT, r.smem, st>>>(r.fa);
            else k_rotate<float, 32><<<r.grid, NT, r.smem, st>>>(r.fa);
            break;
        case OP_LDL:
            if (r.variant == 32) k_ldl_warp<<<r.grid, 32 * LW, r.smem, st>>>(r.fa);
            else if (r.variant == 128) k_ldl<128><<<r.grid, 128, r.smem, st>>>(r.fa, r.flag);
            else k_ldl<NT><<<r.grid, NT, r.smem, st>>>(r.fa, r.flag);
            break;
        case OP_TRSM:
            if (r.variant) k_trsm<float><<<r.grid, NT, r.smem, st>>>(r.fa, r.flag);
            else k_trsm<double><<<r.grid, NT, r.smem, st>>>(r.fa, r.flag);
            break;
        case OP_SCHUR:
            if (r.variant == 1) k_schur_f32<<<r.grid, NT, 0, st>>>(r.sa);
            else if (r.variant == 2) k_schur_oz<<<r.grid, NT, 0, st>>>(r.sa);
            else if (r.variant == 3) k_schur_tc<<<r.grid, TC_THREADS, r.smem, st>>>(r.sa);
            else k_schur<double><<<r.grid, NT, 0, st>>>(r.sa);
            break;
        case OP_MERGE: k_merge<<<r.grid, NT, 0, st>>>(r.ma); break;
        default: r.tiny(st); break;
    }
}

// enqueue one full factorization of the workspace's lanes on stream st;
// returns the number of kernel launches
// Enqueues one batch's kernels on st.  With lookahead (graph captures only),
// the side-branch records go to the handle's second stream between a fork
// (st's progress recorded, the side stream waits for it) and a join (the side
// stream's progress recorded, st waits for it).
static int enqueue_factorization(h2_matrix* h, cudaStream_t st, Profiler* prof, int mixed, bool lookahead = false) {
    FactorState* fs = state_of(h);
    int nl = 0;
    for (const LaunchRec& r : factor_records(h, mixed, lookahead)) {
        if (r.op == OP_FORK) {
            CK(cudaEventRecord(fs->ev_fork, st));
            CK(cudaStreamWaitEvent(fs->side, fs->ev_fork, 0));
            continue;
        }
        if (r.op == OP_JOIN) {
            CK(cudaEventRecord(fs->ev_join, fs->side));
            CK(cudaStreamWaitEvent(st, fs->ev_join, 0));
            continue;
        }
        ++nl;
        if (prof) prof->before(r.kind);
        launch_single(r, r.branch ? fs->side : st);
        if (prof) prof->after();
    }
    return nl;
}

// Autotuning (h2_options.autotune): every candidate of each per-level choice
// (Bunch-Kaufman: one warp, 128 or 256 threads per block; recompression: one
// CTA or a cluster) runs on full batches of shifts spread over the Gershgorin
// interval; each launch is timed with CUDA events on the handle's stream (the
// second of two runs per pass, warm), and every level keeps its fastest
// kernel.
static int autotune(h2_matrix* h) {
    const int L = h->plan.L;
    Workspace& ws = h->ws;
    FactorState* fs = state_of(h);
    cudaStream_t st = h->stream;
    const int mixed = h->opt.precision == H2_PREC_MIXED ? 1 : 0;
    const int LN = ws.lanes;
    std::vector<double> sh(LN);
    for (int i = 0; i < LN; ++i) sh[i] = h->glo + (h->ghi - h->glo) * (i + 0.5) / LN;
    CK(cudaMemcpyAsync(ws.d_shifts, sh.data(), LN * sizeof(double), cudaMemcpyHostToDevice, st));
    k_set_int<<<1, 1, 0, st>>>(fs->d_active, LN);
    // pass c runs LDL candidate c and recompression candidate c % 2
    constexpr int NPASS = 3;
    const int cand_ldl[NPASS] = {32, NT, 128};   // 32: one warp per block (blocks <= 64)
    const int cand_rc[NPASS] = {0, 1, 0};
    std::vector<double> t_ldl[NPASS], t_rc[NPASS];
    for (int c = 0; c < NPASS; ++c) {
        t_ldl[c].assign(L + 1, 0.0);
        t_rc[c].assign(L + 1, 0.0);
        h->tune_ldl.assign(L + 1, cand_ldl[c]);
        h->tune_recomp.assign(L + 1, cand_rc[c]);
        for (int rep = 0; rep < 2; ++rep) {
            std::vector<LaunchRec> recs = factor_records(h, mixed);
            std::vector<cudaEvent_t> ev(2 * recs.size());
            for (auto& e : ev) CK(cudaEventCreate(&e));
            for (size_t i = 0; i < recs.size(); ++i) {
                CK(cudaEventRecord(ev[2 * i], st));
                launch_single(recs[i], st);
                CK(cudaEventRecord(ev[2 * i + 1], st));
            }
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(st));
            for (size_t i = 0; rep == 1 && i < recs.size(); ++i) {
                const LaunchRec& r = recs[i];
                if (r.phase != 2) continue;
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]));
                const int l = L - r.step;
                if (r.op == OP_LDL) t_ldl[c][l] += t;
                if (r.op == OP_RECOMP || r.op == OP_RECOMP_CL) t_rc[c][l] += t;
            }
            for (auto& e : ev) cudaEventDestroy(e);
        }
    }
    for (int l = 0; l <= L; ++l) {
        int bl = 0;
        for (int c = 1; c < NPASS; ++c)
            if (t_ldl[c][l] < t_ldl[bl][l]) bl = c;
        h->tune_ldl[l] = cand_ldl[bl];
        const double t0 = std::min(t_rc[0][l], t_rc[2][l]);
        h->tune_recomp[l] = t0 <= t_rc[1][l] ? cand_rc[0] : cand_rc[1];
    }
    CK(cudaMemsetAsync(ws.d_err, 0, 8 * sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    return H2_OK;
}

int tune_choice(h2_matrix* h, int level, int* out) {
    const int Dm = h->lev[level].dmax;
    const LevelWork& W = state_of(h)->lw[level];
    const int nfm = W.colours.empty() ? 0 : W.colours[0].nfill_max;
    out[0] = ldl_threads(h, level, Dm);
    out[1] = recomp_clustered(h, level, nfm, Dm) ? 1 : 0;
    return H2_OK;
}

// ------------------------------------------------------------ groups --
// A group runs one batch for several handles: records of equal key from all
// handles become one grouped launch (GroupArgs tables), so every level
// (counted from the leaves) and colour is one launch over all matrices.
struct GLaunch {
    int op = 0, variant = 0, block = NT;
    size_t smem = 0;
    unsigned gx = 0, gy = 0;
    void* d_args = nullptr;
    int* d_off = nullptr;
    int* d_flag = nullptr;
    int n = 0;
    std::vector<const LaunchRec*> tiny;
};

}  // namespace h2

struct h2_group_set {
    std::vector<h2_matrix*> hs;
    cudaStream_t stream = nullptr;
    int lanes = 0, mixed = 0;
    std::vector<std::vector<h2::LaunchRec>> recs;     // per handle, batch precision
    std::vector<std::vector<h2::LaunchRec>> recs64;   // mixed groups: the FP64 re-run batch
    std::vector<h2::GLaunch> launches, launches64;
    std::vector<void*> dev;
    cudaGraphExec_t graph = nullptr;
    cudaGraphExec_t graph64 = nullptr;
};

namespace h2 {

template <typename Args>
static int upload_items(h2_group_set* g, const std::vector<const LaunchRec*>& items, Args LaunchRec::*member,
                        GLaunch& gl) {
    std::vector<Args> args;
    std::vector<int> off(1, 0), flag;
    for (const LaunchRec* r : items) {
        args.push_back(r->*member);
        off.push_back(off.back() + (int)r->grid.x);
        flag.push_back(r->flag);
    }
    int rc;
    Args* da = nullptr;
    int* doff = nullptr;
    int* dflag = nullptr;
    if ((rc = dalloc(&da, args.size())) || (rc = dalloc(&doff, off.size())) || (rc = dalloc(&dflag, flag.size())))
        return rc;
    g->dev.push_back(da);
    g->dev.push_back(doff);
    g->dev.push_back(dflag);
    CK(cudaMemcpy(da, args.data(), args.size() * sizeof(Args), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(doff, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dflag, flag.data(), flag.size() * sizeof(int), cudaMemcpyHostToDevice));
    gl.d_args = da;
    gl.d_off = doff;
    gl.d_flag = dflag;
    gl.n = (int)items.size();
    gl.gx = (unsigned)off.back();
    return H2_OK;
}

static void launch_grouped(const GLaunch& gl, cudaStream_t st) {
    const dim3 grid(gl.gx, gl.gy);
    GroupArgs<FactorArgs> F{(const FactorArgs*)gl.d_args, gl.d_off, gl.d_flag, gl.n};
    GroupArgs<SchurArgs> S{(const SchurArgs*)gl.d_args, gl.d_off, gl.d_flag, gl.n};
    switch (gl.op) {
        case OP_INIT_LEAF:
            k_init_leaf_g<<<grid, NT, 0, st>>>(GroupArgs<InitArgs>{(const InitArgs*)gl.d_args, gl.d_off, gl.d_flag, gl.n});
            break;
        case OP_RECOMP: k_recomp_g<<<grid, NT, 0, st>>>(F); break;
        case OP_RECOMP_CL: k_recomp_cluster_g<<<grid, NT, gl.smem, st>>>(F); break;
        case OP_ROTATE:
            if (gl.variant == 0) k_rotate_fp64_g<<<grid, NT, gl.smem, st>>>(F);
            else if (gl.variant == 2) k_rotate_oz_g<<<grid, NT, gl.smem, st>>>(F);
            else if (gl.variant == 8) k_rotate_g<float, 8><<<grid, NT, gl.smem, st>>>(F);
            else if (gl.variant == 16) k_rotate_g<float, 16><<<grid, NT, gl.smem, st>>>(F);
            else k_rotate_g<float, 32><<<grid, NT, gl.smem, st>>>(F);
            break;
        case OP_LDL:
            if (gl.variant == 32) k_ldl_warp_g<<<grid, 32 * LW, gl.smem, st>>>(F);
            else if (gl.variant == 128) k_ldl_g<128><<<grid, 128, gl.smem, st>>>(F);
            else k_ldl_g<NT><<<grid, NT, gl.smem, st>>>(F);
            break;
        case OP_TRSM:
            if (gl.variant) k_trsm_g<float><<<grid, NT, gl.smem, st>>>(F);
            else k_trsm_g<double><<<grid, NT, gl.smem, st>>>(F);
            break;
        case OP_SCHUR:
            if (gl.variant == 1) k_schur_f32_g<<<grid, NT, 0, st>>>(S);
            else if (gl.variant == 2) k_schur_oz_g<<<grid, NT, 0, st>>>(S);
            else if (gl.variant == 3) k_schur_tc_g<<<grid, TC_THREADS, gl.smem, st>>>(S);
            else k_schur_g<double><<<grid, NT, 0, st>>>(S);
            break;
        case OP_MERGE:
            k_merge_g<<<grid, NT, 0, st>>>(GroupArgs<MergeArgs>{(const MergeArgs*)gl.d_args, gl.d_off, gl.d_flag, gl.n});
            break;
        default:
            for (const LaunchRec* r : gl.tiny) r->tiny(st);
            break;
    }
}

void group_destroy(h2_group_set* g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->graph) cudaGraphExecDestroy(g->graph);
    if (g->graph64) cudaGraphExecDestroy(g->graph64);
    for (void* p : g->dev) cudaFree(p);
    delete g;
}

// The grouped launches of one batch precision over all handles of g (records
// of equal (phase, step, colour, op, variant) merged) and their CUDA graph.
static int group_graph(h2_group_set* g, int mixed, std::vector<std::vector<LaunchRec>>& recs,
                       std::vector<GLaunch>& launches, cudaGraphExec_t* ge) {
    const int nh = (int)g->hs.size();
    struct Ref {
        const LaunchRec* r;
        int h;
    };
    std::vector<Ref> all;
    recs.resize(nh);
    for (int i = 0; i < nh; ++i) recs[i] = factor_records(g->hs[i], mixed);
    for (int i = 0; i < nh; ++i)
        for (const LaunchRec& r : recs[i]) all.push_back(Ref{&r, i});
    auto key = [](const LaunchRec* r) {
        return std::make_tuple(r->phase, r->step, r->colour, r->op, r->variant);
    };
    std::stable_sort(all.begin(), all.end(), [&](const Ref& a, const Ref& b) { return key(a.r) < key(b.r); });
    int rc;
    for (size_t i = 0; i < all.size();) {
        size_t j = i;
        std::vector<const LaunchRec*> items;
        while (j < all.size() && key(all[j].r) == key(all[i].r)) items.push_back(all[j++].r);
        const LaunchRec* r0 = items[0];
        GLaunch gl;
        gl.op = r0->op;
        gl.variant = r0->variant;
        gl.block = r0->block;
        gl.gy = r0->grid.y;
        for (const LaunchRec* r : items) gl.smem = std::max(gl.smem, r->smem);
        rc = H2_OK;
        switch (r0->op) {
            case OP_INIT_LEAF: rc = upload_items(g, items, &LaunchRec::ia, gl); break;
            case OP_SCHUR: rc = upload_items(g, items, &LaunchRec::sa, gl); break;
            case OP_MERGE: rc = upload_items(g, items, &LaunchRec::ma, gl); break;
            case OP_RECOMP: case OP_RECOMP_CL: case OP_ROTATE: case OP_LDL: case OP_TRSM:
                rc = upload_items(g, items, &LaunchRec::fa, gl);
                break;
            default: gl.tiny = items; break;
        }
        if (rc) return rc;
        launches.push_back(gl);
        i = j;
    }
    // one graph for the whole group batch
    cudaStream_t st = g->stream;
    cudaGraph_t graph;
    CK(cudaStreamSynchronize(st));
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    for (const GLaunch& gl : launches) launch_grouped(gl, st);
    CK(cudaStreamEndCapture(st, &graph));
    CK(cudaGraphInstantiate(ge, graph, 0));
    cudaGraphDestroy(graph);
    return H2_OK;
}

int group_create(h2_matrix* const* hs, int nh, h2_group_set** out) {
    auto* g = new h2_group_set();
    g->hs.assign(hs, hs + nh);
    g->stream = hs[0]->stream;
    g->lanes = hs[0]->ws.lanes;
    g->mixed = hs[0]->opt.precision == H2_PREC_MIXED ? 1 : 0;
    for (h2_matrix* h : g->hs)
        if (h->ws.lanes != g->lanes || h->opt.precision != hs[0]->opt.precision) {
            delete g;
            set_error("h2_group_create: handles need equal max_lanes and precision");
            return H2_ERR_INVALID_ARG;
        }
    CK(cudaFuncSetAttribute(k_rotate_fp64_g, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    CK(cudaFuncSetAttribute(k_rotate_oz_g, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    CK(cudaFuncSetAttribute(k_rotate_g<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    CK(cudaFuncSetAttribute(k_rotate_g<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    CK(cudaFuncSetAttribute(k_rotate_g<float, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    CK(cudaFuncSetAttribute(k_ldl_g<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap + 8192));
    CK(cudaFuncSetAttribute(k_ldl_warp_g, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    CK(cudaFuncSetAttribute(k_ldl_g<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap + 8192));
    CK(cudaFuncSetAttribute(k_trsm_g<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap + 8192));
    CK(cudaFuncSetAttribute(k_trsm_g<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap + 8192));
    CK(cudaFuncSetAttribute(k_schur_tc_g, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    int rc = group_graph(g, g->mixed, g->recs, g->launches, &g->graph);
    if (rc == H2_OK && g->mixed) rc = group_graph(g, 0, g->recs64, g->launches64, &g->graph64);
    if (rc) {
        group_destroy(g);
        return rc;
    }
    *out = g;
    return H2_OK;
}

int group_launches(const h2_group_set* g) {
    int n = 0;
    for (const GLaunch& gl : g->launches) n += gl.tiny.empty() ? 1 : (int)gl.tiny.size();
    return n;
}

int group_inertia(h2_group_set* g, const double* d_shifts, const int* ns, int64_t* d_counts, double* d_minpiv) {
    const int nh = (int)g->hs.size(), LN = g->lanes;
    cudaStream_t st = g->stream;
    for (int i = 0; i < nh; ++i)
        if (ns[i] < 0 || ns[i] > LN) {
            set_error("h2_group_inertia_device: ns outside 0..max_lanes");
            return H2_ERR_INVALID_ARG;
        }
    if (g->mixed) {
        // certified counts (k_guard_certify): mixed group batches of
        // (mu - Delta, mu + Delta) pairs, then one FP64 group batch of the
        // shifts left uncertified, all handles together, no host round trip
        int nsmax = 0;
        for (int i = 0; i < nh; ++i) {
            h2_matrix* h = g->hs[i];
            FactorState* fs = state_of(h);
            nsmax = std::max(nsmax, ns[i]);
            if (ns[i] > 0)
                CK(cudaMemcpyAsync(fs->d_req, d_shifts + (size_t)i * LN, ns[i] * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
            k_set_int<<<1, 1, 0, st>>>(fs->d_rr_n, 0);
        }
        const int half = LN / 2;
        if (half < 1) {
            for (int i = 0; i < nh; ++i) {
                FactorState* fs = state_of(g->hs[i]);
                k_guard_all<<<1, 256, 0, st>>>(ns[i], fs->d_rr_idx, fs->d_rr_n, fs->d_tally);
            }
        } else {
            for (int c0 = 0; c0 < nsmax; c0 += half) {
                for (int i = 0; i < nh; ++i) {
                    const int nc = std::max(0, std::min(half, ns[i] - c0));
                    if (nc > 0) guard_pairs(g->hs[i], c0, nc);
                    else k_set_int<<<1, 1, 0, st>>>(state_of(g->hs[i])->d_active, 0);
                }
                CK(cudaGraphLaunch(g->graph, st));
                for (int i = 0; i < nh; ++i) {
                    const int nc = std::max(0, std::min(half, ns[i] - c0));
                    if (nc > 0) guard_certify(g->hs[i], c0, nc);
                }
            }
        }
        for (int i = 0; i < nh; ++i) guard_rerun_setup(g->hs[i]);
        CK(cudaGraphLaunch(g->graph64, st));
        for (int i = 0; i < nh; ++i) {
            if (ns[i] == 0) continue;
            h2_matrix* h = g->hs[i];
            FactorState* fs = state_of(h);
            guard_scatter(h);
            CK(cudaMemcpyAsync(d_counts + (size_t)i * LN, fs->d_gc, ns[i] * sizeof(int64_t),
                               cudaMemcpyDeviceToDevice, st));
            if (d_minpiv)
                CK(cudaMemcpyAsync(d_minpiv + (size_t)i * LN, fs->d_gmp, ns[i] * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
        }
        CK(cudaGetLastError());
        return H2_OK;
    }
    for (int i = 0; i < nh; ++i) {
        h2_matrix* h = g->hs[i];
        if (ns[i] > 0)
            CK(cudaMemcpyAsync(h->ws.d_shifts, d_shifts + (size_t)i * LN, ns[i] * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
        k_set_int<<<1, 1, 0, st>>>(state_of(h)->d_active, ns[i]);
    }
    CK(cudaGraphLaunch(g->graph, st));
    for (int i = 0; i < nh; ++i) {
        if (ns[i] == 0) continue;
        FactorState* fs = state_of(g->hs[i]);
        CK(cudaMemcpyAsync(d_counts + (size_t)i * LN, fs->d_counts, ns[i] * sizeof(int64_t),
                           cudaMemcpyDeviceToDevice, st));
        if (d_minpiv)
            CK(cudaMemcpyAsync(d_minpiv + (size_t)i * LN, fs->d_mp, ns[i] * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaGetLastError());
    return H2_OK;
}

static int ensure_graph(h2_matrix* h, int mixed) {
    Workspace& ws = h->ws;
    cudaGraphExec_t& ge = mixed ? ws.graph_mixed : ws.graph;
    if (ge) return H2_OK;
    cudaStream_t st = h->stream;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    h->kernels_per_batch = enqueue_factorization(h, st, nullptr, mixed, lookahead_on(h));
    CK(cudaStreamEndCapture(st, &g));
    CK(cudaGraphInstantiate(&ge, g, 0));
    cudaGraphDestroy(g);
    return H2_OK;
}

// launch one batch of the lanes already in ws.d_shifts (count set on device):
// replay the captured graph, or launch the same kernels one by one
static int launch_batch(h2_matrix* h, int mixed) {
    if (!use_graphs(h)) {
        h->kernels_per_batch = enqueue_factorization(h, h->stream, nullptr, mixed);
        CK(cudaGetLastError());
        return H2_OK;
    }
    int rc = ensure_graph(h, mixed);
    if (rc) return rc;
    CK(cudaGraphLaunch(mixed ? h->ws.graph_mixed : h->ws.graph, h->stream));
    return H2_OK;
}

// Delta of the mixed-precision guard: 64 u_32 ||A||_inf, about 200 times the
// measured ||E|| of the FP32 products at n = 1024
static double guard_delta(const h2_matrix* h) { return 64.0 * 0x1.0p-24 * h->norm_inf; }

// Guard steps of one handle (see k_guard_certify).  Pairs of chunk c0 .. of
// the shifts in fs->d_req, before the mixed batch of that chunk:
static void guard_pairs(h2_matrix* h, int c0, int nc) {
    FactorState* fs = state_of(h);
    k_guard_pairs<<<(nc + 255) / 256, 256, 0, h->stream>>>(fs->d_req + c0, nc, guard_delta(h), h->ws.d_shifts,
                                                           fs->d_active);
}
static void guard_certify(h2_matrix* h, int c0, int nc) {
    FactorState* fs = state_of(h);
    k_guard_certify<<<1, 1024, 0, h->stream>>>(fs->d_counts, fs->d_mp, nc, c0, h->opt.pivot_guard * h->norm_inf,
                                               fs->d_gc, fs->d_gmp, fs->d_rr_idx, fs->d_rr_n, fs->d_tally);
}
static void guard_rerun_setup(h2_matrix* h) {
    FactorState* fs = state_of(h);
    const int LN = h->ws.lanes;
    k_guard_rerun_setup<<<(LN + 255) / 256, 256, 0, h->stream>>>(fs->d_req, fs->d_rr_idx, fs->d_rr_n,
                                                                 h->ws.d_shifts, fs->d_active);
}
static void guard_scatter(h2_matrix* h) {
    FactorState* fs = state_of(h);
    const int LN = h->ws.lanes;
    k_guard_scatter<<<(LN + 255) / 256, 256, 0, h->stream>>>(fs->d_rr_idx, fs->d_rr_n, fs->d_counts, fs->d_mp,
                                                             fs->d_gc, fs->d_gmp);
}

// Certified mixed-precision counts of the ns shifts in fs->d_req into
// fs->d_gc / fs->d_gmp, all on the handle's stream: mixed batches of
// (mu - Delta, mu + Delta) pairs, lanes / 2 shifts each, then one FP64 batch
// of the shifts left uncertified.  No host round trip.
static int enqueue_guarded(h2_matrix* h, int ns) {
    FactorState* fs = state_of(h);
    cudaStream_t st = h->stream;
    const int half = h->ws.lanes / 2;
    int rc;
    k_set_int<<<1, 1, 0, st>>>(fs->d_rr_n, 0);
    if (half < 1) {
        k_guard_all<<<1, 256, 0, st>>>(ns, fs->d_rr_idx, fs->d_rr_n, fs->d_tally);
    } else {
        for (int c0 = 0; c0 < ns; c0 += half) {
            const int nc = std::min(half, ns - c0);
            guard_pairs(h, c0, nc);
            if ((rc = launch_batch(h, 1))) return rc;
            guard_certify(h, c0, nc);
        }
    }
    guard_rerun_setup(h);
    if ((rc = launch_batch(h, 0))) return rc;
    guard_scatter(h);
    CK(cudaGetLastError());
    return H2_OK;
}

int run_inertia(h2_matrix* h, const double* d_shifts, int ns, int64_t* d_counts, double* d_minpiv) {
    Workspace& ws = h->ws;
    FactorState* fs = state_of(h);
    cudaStream_t st = h->stream;
    if (ns <= 0) return H2_OK;
    if (ns > ws.lanes) {
        set_error("h2_inertia_device: ns exceeds max_lanes");
        return H2_ERR_INVALID_ARG;
    }
    const int mixed = h->opt.precision == H2_PREC_MIXED;
    int rc = use_graphs(h) ? ensure_graph(h, mixed) : H2_OK;
    if (rc) return rc;
    if (mixed) {
        CK(cudaMemcpyAsync(fs->d_req, d_shifts, ns * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if ((rc = enqueue_guarded(h, ns))) return rc;
        CK(cudaMemcpyAsync(d_counts, fs->d_gc, ns * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
        if (d_minpiv) CK(cudaMemcpyAsync(d_minpiv, fs->d_gmp, ns * sizeof(double), cudaMemcpyDeviceToDevice, st));
        return H2_OK;
    }
    CK(cudaMemcpyAsync(ws.d_shifts, d_shifts, ns * sizeof(double), cudaMemcpyDeviceToDevice, st));
    k_set_int<<<1, 1, 0, st>>>(fs->d_active, ns);
    if ((rc = launch_batch(h, 0))) return rc;
    CK(cudaMemcpyAsync(d_counts, fs->d_counts, ns * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    if (d_minpiv) CK(cudaMemcpyAsync(d_minpiv, fs->d_mp, ns * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return H2_OK;
}

int guard_tally(h2_matrix* h, int64_t* checked, int64_t* rerun) {
    unsigned long long t[2] = {0, 0};
    CK(cudaMemcpyAsync(t, state_of(h)->d_tally, sizeof(t), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *checked = (int64_t)t[0];
    *rerun = (int64_t)t[1];
    return H2_OK;
}

std::string err_message(const int* e) {
    if (e[0] & 2)
        return "kernel " + std::to_string(e[1]) + " met out-of-range sizes (" + std::to_string(e[2]) + ", " +
               std::to_string(e[3]) + ", " + std::to_string(e[4]) + ", " + std::to_string(e[5]) + ") at block (" +
               std::to_string(e[6]) + ", " + std::to_string(e[7]) + ") and skipped its work";
    return "NaN pivot in the factorization";
}

// heartbeat buffer (host side), set up once per process when H2_HEARTBEAT=1
static unsigned int* g_hb_host = nullptr;

int heartbeat_setup() {
    const char* e = getenv("H2_HEARTBEAT");
    if (!e || e[0] != '1' || g_hb_host) return H2_OK;
    CK(cudaHostAlloc((void**)&g_hb_host, 64 * sizeof(unsigned int), cudaHostAllocMapped));
    std::memset(g_hb_host, 0, 64 * sizeof(unsigned int));
    unsigned int* d = nullptr;
    CK(cudaHostGetDevicePointer((void**)&d, g_hb_host, 0));
    CK(cudaMemcpyToSymbol(g_hb, &d, sizeof(d)));
    return H2_OK;
}

void heartbeat_read(unsigned int* out) {
    for (int i = 0; i < 64; ++i) out[i] = g_hb_host ? ((volatile unsigned int*)g_hb_host)[i] : 0u;
}

int run_status(h2_matrix* h, int64_t* info) {
    int e[8] = {0};
    CK(cudaMemcpyAsync(e, h->ws.d_err, sizeof(e), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemsetAsync(h->ws.d_err, 0, sizeof(e), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < 8; ++i) info[i] = e[i];
    if (e[0]) {
        set_error(err_message(e));
        return H2_ERR_NUMERICAL;
    }
    return H2_OK;
}

// one batch of host shifts (nb <= lanes) in the given precision; counts and
// min |pivot| back to host arrays
static int host_batch(h2_matrix* h, const double* shifts, int nb, int mixed, int64_t* counts, double* minpiv) {
    Workspace& ws = h->ws;
    FactorState* fs = state_of(h);
    cudaStream_t st = h->stream;
    CK(cudaMemcpyAsync(ws.d_shifts, shifts, nb * sizeof(double), cudaMemcpyHostToDevice, st));
    k_set_int<<<1, 1, 0, st>>>(fs->d_active, nb);
    int rc = launch_batch(h, mixed);
    if (rc) return rc;
    CK(cudaMemcpyAsync(counts, fs->d_counts, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(minpiv, fs->d_mp, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    int err[8] = {0};
    CK(cudaMemcpyAsync(err, ws.d_err, sizeof(err), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err[0]) {
        set_error(err_message(err));
        return H2_ERR_NUMERICAL;
    }
    return H2_OK;
}

// mixed precision, host arrays: one batch of nb <= lanes shifts through the
// certified device path (enqueue_guarded)
static int host_batch_guarded(h2_matrix* h, const double* shifts, int nb, int64_t* counts, double* minpiv) {
    Workspace& ws = h->ws;
    FactorState* fs = state_of(h);
    cudaStream_t st = h->stream;
    CK(cudaMemcpyAsync(fs->d_req, shifts, nb * sizeof(double), cudaMemcpyHostToDevice, st));
    int rc = enqueue_guarded(h, nb);
    if (rc) return rc;
    CK(cudaMemcpyAsync(counts, fs->d_gc, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(minpiv, fs->d_gmp, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    int err[8] = {0};
    CK(cudaMemcpyAsync(err, ws.d_err, sizeof(err), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err[0]) {
        set_error(err_message(err));
        return H2_ERR_NUMERICAL;
    }
    return H2_OK;
}

int run_profile(h2_matrix* h, const double* d_shifts, int ns, int64_t* d_counts, double* ms,
                int64_t* launches, double* flops, double* bytes) {
    Workspace& ws = h->ws;
    FactorState* fs = state_of(h);
    cudaStream_t st = h->stream;
    if (ns <= 0 || ns > ws.lanes) {
        set_error("h2_profile_batch: need 1 <= ns <= max_lanes");
        return H2_ERR_INVALID_ARG;
    }
    CK(cudaMemcpyAsync(ws.d_shifts, d_shifts, ns * sizeof(double), cudaMemcpyDeviceToDevice, st));
    k_set_int<<<1, 1, 0, st>>>(fs->d_active, ns);
    Profiler pr;
    pr.st = st;
    int nl = enqueue_factorization(h, st, &pr, h->opt.precision == H2_PREC_MIXED);
    CK(cudaMemcpyAsync(d_counts, fs->d_counts, ns * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    double stats[2 * H2_NKINDS];
    CK(cudaMemcpyAsync(stats, fs->d_stats, sizeof(stats), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int k = 0; k < H2_NKINDS; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
        flops[k] = stats[k];
        bytes[k] = stats[H2_NKINDS + k];
    }
    for (size_t i = 0; i < pr.kind.size(); ++i) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, pr.ev[2 * i], pr.ev[2 * i + 1]));
        ms[pr.kind[i]] += t;
        launches[pr.kind[i]] += 1;
    }
    for (auto e : pr.ev) cudaEventDestroy(e);
    (void)nl;
    return H2_OK;
}

// host arrays: each batch of <= lanes shifts is copied in, factorized and its
// counts copied back (the end-to-end path of h2_inertia); in mixed precision
// the guarded shifts of each batch are re-run in FP64
int run_inertia_host(h2_matrix* h, const double* shifts, int64_t ns, int64_t* counts, double* minpiv) {
    Workspace& ws = h->ws;
    cudaStream_t st = h->stream;
    const int mixed = h->opt.precision == H2_PREC_MIXED;
    CK(cudaMemsetAsync(ws.d_err, 0, 8 * sizeof(int), st));
    std::vector<double> mp(ws.lanes);
    for (int64_t b0 = 0; b0 < ns; b0 += ws.lanes) {
        int nb = (int)std::min<int64_t>(ws.lanes, ns - b0);
        int rc = mixed ? host_batch_guarded(h, shifts + b0, nb, counts + b0, mp.data())
                       : host_batch(h, shifts + b0, nb, 0, counts + b0, mp.data());
        if (rc) return rc;
        if (minpiv) std::memcpy(minpiv + b0, mp.data(), nb * sizeof(double));
    }
    return H2_OK;
}

// --------------------------------------------------------------- bisection --
// plan: distinct active intervals get the lanes; each gets q points
// lo + (hi-lo) j/(q+1), j = 1..q
// Plan of one multisection round over nk brackets sorted by k.  Brackets of
// sorted k narrowed by the same (mu, nu) pairs are monotone in k, so equal
// brackets are adjacent and the first of each run is a distinct interval (a
// missed duplicate would only repeat work).  One CTA scans the brackets in
// chunks (block prefix sums), keeps the first `lanes` distinct intervals
// wider than tol in k order and spreads the lanes over them: interval u gets
// q or q + 1 equally spaced interior points.  per > 0 caps the round at per
// shifts per interval: with few intervals, a round of fewer lanes is cheaper
// by more than the fewer bits of narrowing it gives (one k at n = 1024: 16
// shifts per round beat 64).
__device__ __forceinline__ void bisect_plan_body(const double* lo, const double* hi, int nk, double tol, int lanes,
                                                 int per, double* shifts, int* active, int* nact, int* first) {
    __shared__ int wsum[32];
    __shared__ int s_base;
    const int t = threadIdx.x, w = t >> 5, l = t & 31, nw = (blockDim.x + 31) >> 5;
    if (t == 0) s_base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nk; c0 += blockDim.x) {
        const int k = c0 + t;
        int f = 0;
        if (k < nk && hi[k] - lo[k] >= tol) f = (k == 0 || !(lo[k - 1] == lo[k] && hi[k - 1] == hi[k])) ? 1 : 0;
        int incl = f;                                   // inclusive scan within the warp
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (l >= o) incl += v;
        }
        if (l == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            int v = l < nw ? wsum[l] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, v, o);
                if (l >= o) v += u;
            }
            if (l < nw) wsum[l] = v;                    // inclusive warp prefix
        }
        __syncthreads();
        const int before = s_base + (w > 0 ? wsum[w - 1] : 0) + incl - f;
        if (f && before < lanes) first[before] = k;
        __syncthreads();
        if (t == 0) s_base += wsum[nw - 1];
        __syncthreads();
    }
    const int nd = s_base;
    const int use = (per > 0 && nd > 0) ? (int)min((long long)lanes, (long long)nd * per) : lanes;
    if (t == 0) {
        *nact = nd;
        *active = nd > 0 ? use : 0;
    }
    const int m = min(nd, use);
    if (m == 0) return;
    const int q = use / m, extra = use % m;
    for (int u = t; u < m; u += blockDim.x) {
        const int qu = q + (u < extra ? 1 : 0);
        const int off = u * q + min(u, extra);
        const int k = first[u];
        const double a = lo[k], b = hi[k];
        for (int j = 1; j <= qu; ++j) shifts[off + j - 1] = a + (b - a) * (double)j / (double)(qu + 1);
    }
}

__global__ void __launch_bounds__(1024) k_bisect_plan(const double* lo, const double* hi, int nk, double tol,
                                                      int lanes, int per, double* shifts, int* active, int* nact,
                                                      int* first) {
    bisect_plan_body(lo, hi, nk, tol, lanes, per, shifts, active, nact, first);
}


// The plan step of one loop iteration: as k_bisect_plan, then the loop's
// condition -- continue while some interval is wider than the width and the
// round cap is not reached (one thread sets it).
__global__ void __launch_bounds__(1024) k_bisect_plan_loop(const double* lo, const double* hi, KthLoop* par,
                                                           int lanes, double* shifts, int* active, int* nact,
                                                           int* first, cudaGraphConditionalHandle cond) {
    const int nk = par->nk;
    bisect_plan_body(lo, hi, nk, par->width, lanes, par->per_interval, shifts, active, nact, first);
    if (threadIdx.x == 0) {
        const int nd = *nact;
        int go = nd > 0 ? 1 : 0;
        if (go) {
            par->rounds += 1;
            par->shifts += (unsigned long long)*active;
            if (par->rounds >= par->max_rounds) {
                par->stopped = 1;
                go = 0;
            }
        }
        cudaGraphSetConditional(cond, go);
    }
}

__global__ void k_bisect_update_loop(double* lo, double* hi, const int64_t* kk, const KthLoop* par,
                                     const double* shifts, const int64_t* counts, const int* active) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= par->nk) return;
    double a = lo[k], b = hi[k];
    const int64_t kv = kk[k];
    const int ns = *active;
    for (int i = 0; i < ns; ++i) {
        const double mu = shifts[i];
        if (a < mu && mu < b) {
            if (counts[i] >= kv) b = mu;
            else a = mu;
        }
    }
    lo[k] = a;
    hi[k] = b;
}

__global__ void k_bisect_update(double* lo, double* hi, const int64_t* kk, int nk, const double* shifts,
                                const int64_t* counts, const int* active) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    double a = lo[k], b = hi[k];
    int64_t kv = kk[k];
    int ns = *active;
    for (int i = 0; i < ns; ++i) {
        double mu = shifts[i];
        if (a < mu && mu < b) {
            if (counts[i] >= kv) b = mu;
            else a = mu;
        }
    }
    lo[k] = a;
    hi[k] = b;
}

// One multisection round on the device-resident intervals: plan the shifts of
// the distinct intervals wider than `width`, factorize them in the given
// precision and narrow every k.  h2_kth_eig runs its mixed rounds without the
// per-shift guard: a wrong mixed count at mu implies |lambda_k - mu| < ||E||
// << Delta, so the FP64 check of the widened bracket certifies the result.
// Returns the number of active intervals (0: nothing to do) in *nact.
static int kth_round(h2_matrix* h, int nk, double width, int mixed, int* nact) {
    Workspace& ws = h->ws;
    FactorState* fs = state_of(h);
    cudaStream_t st = h->stream;
    k_bisect_plan<<<1, 1024, 0, st>>>(fs->d_lo, fs->d_hi, nk, width, ws.lanes, h->opt.shifts_per_interval,
                                      ws.d_shifts, fs->d_active, fs->d_nact, fs->d_first);
    int used = 0;
    CK(cudaMemcpyAsync(nact, fs->d_nact, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&used, fs->d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (*nact == 0) return H2_OK;
    int rc = launch_batch(h, mixed);
    if (rc) return rc;
    k_bisect_update<<<(unsigned)((nk + 127) / 128), 128, 0, st>>>(fs->d_lo, fs->d_hi, fs->d_k, nk, ws.d_shifts,
                                                                 fs->d_counts, fs->d_active);
    h->last_shifts += used;
    return H2_OK;
}

// The whole bisection of one precision phase as one CUDA graph: a WHILE
// conditional node whose body is plan (sets the condition), the batch's
// kernels, and the bracket update.  The loop stops on the device when no
// interval is wider than the width (or at the round cap), so a phase costs
// one launch and one wait instead of one host round trip per round.
static int build_loop_graph(h2_matrix* h, int mixed) {
    Workspace& ws = h->ws;
    FactorState* fs = state_of(h);
    cudaStream_t st = h->stream;
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    k_bisect_plan_loop<<<1, 1024, 0, st>>>(fs->d_lo, fs->d_hi, fs->d_loop, ws.lanes, ws.d_shifts, fs->d_active,
                                           fs->d_nact, fs->d_first, cond);
    enqueue_factorization(h, st, nullptr, mixed, lookahead_on(h));
    k_bisect_update_loop<<<(unsigned)((fs->nk_cap + 127) / 128), 128, 0, st>>>(
        fs->d_lo, fs->d_hi, fs->d_k, fs->d_loop, ws.d_shifts, fs->d_counts, fs->d_active);
    cudaGraph_t captured;
    CK(cudaStreamEndCapture(st, &captured));
    CK(cudaGraphInstantiate(&fs->loop_exec[mixed], g, 0));
    cudaGraphDestroy(g);
    return H2_OK;
}

// runs bisection rounds on the device until every bracket is narrower than
// `width`; adds the rounds and shifts to the handle's counters
static int run_loop(h2_matrix* h, int nk, double width, int mixed, int* rounds) {
    FactorState* fs = state_of(h);
    cudaStream_t st = h->stream;
    if (fs->loop_nk_cap != fs->nk_cap) {
        for (auto& e : fs->loop_exec)
            if (e) {
                cudaGraphExecDestroy(e);
                e = nullptr;
            }
        fs->loop_nk_cap = fs->nk_cap;
    }
    int rc;
    if (!fs->loop_exec[mixed] && (rc = build_loop_graph(h, mixed))) return rc;
    KthLoop par{nk, width, 4096, 0, 0ull, 0, h->opt.shifts_per_interval};
    CK(cudaMemcpyAsync(fs->d_loop, &par, sizeof(par), cudaMemcpyHostToDevice, st));
    CK(cudaGraphLaunch(fs->loop_exec[mixed], st));
    CK(cudaMemcpyAsync(&par, fs->d_loop, sizeof(par), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *rounds = par.rounds;
    h->last_shifts += (int64_t)par.shifts;
    if (par.stopped) {
        set_error("h2_kth_eig: bisection did not converge within 4096 rounds");
        return H2_ERR_NUMERICAL;
    }
    return H2_OK;
}

int run_kth(h2_matrix* h, const int64_t* k, int64_t nk, double tol, double* out, double* err_bound,
            const double* interval) {
    Workspace& ws = h->ws;
    FactorState* fs = state_of(h);
    cudaStream_t st = h->stream;
    int rc;
    // brackets in k order (equal brackets adjacent, see k_bisect_plan); the
    // results go back to the caller's order
    std::vector<int64_t> order(nk), ks(nk);
    for (int64_t i = 0; i < nk; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return k[x] < k[y]; });
    for (int64_t i = 0; i < nk; ++i) ks[i] = k[order[i]];
    k = ks.data();
    CK(cudaMemsetAsync(ws.d_err, 0, 8 * sizeof(int), st));
    // start interval: the caller's [a, b] with nu(a) < k <= nu(b) for every k
    // (checked in FP64), else the Gershgorin interval padded by 1e-6 ||A||_inf
    // with nu(a) = 0 and nu(b) = n (checked)
    const double a = interval ? interval[0] : h->glo - 1e-6 * h->norm_inf;
    const double b = interval ? interval[1] : h->ghi + 1e-6 * h->norm_inf;
    int64_t nu_a = 0, nu_b = h->n;
    if (ws.lanes >= 2 || interval) {
        double sh[2] = {a, b}, mp[2];
        int64_t cnt[2] = {0, 0};
        if (ws.lanes >= 2) {
            if ((rc = host_batch(h, sh, 2, 0, cnt, mp))) return rc;
        } else if ((rc = host_batch(h, sh, 1, 0, cnt, mp)) || (rc = host_batch(h, sh + 1, 1, 0, cnt + 1, mp + 1))) {
            return rc;
        }
        if (interval) {
            nu_a = cnt[0];
            nu_b = cnt[1];
            if (!(nu_a < k[0] && k[nk - 1] <= nu_b)) {
                set_error("h2_kth_eig_in: the interval does not hold every requested eigenvalue (nu(lo) = " +
                          std::to_string(nu_a) + ", nu(hi) = " + std::to_string(nu_b) + ")");
                return H2_ERR_INTERVAL;
            }
        } else if (cnt[0] != 0 || cnt[1] != h->n) {
            set_error("h2_kth_eig: nu(a) != 0 or nu(b) != n on the Gershgorin interval");
            return H2_ERR_INTERVAL;
        }
    }
    if (fs->nk_cap < nk) {
        cudaFree(fs->d_lo); cudaFree(fs->d_hi); cudaFree(fs->d_k); cudaFree(fs->d_nact); cudaFree(fs->d_first);
        fs->d_lo = fs->d_hi = nullptr;
        fs->d_k = nullptr;
        fs->d_nact = fs->d_first = nullptr;
        fs->nk_cap = 0;
        if ((rc = dalloc(&fs->d_lo, nk)) || (rc = dalloc(&fs->d_hi, nk)) || (rc = dalloc(&fs->d_k, nk)) ||
            (rc = dalloc(&fs->d_nact, 1)) || (rc = dalloc(&fs->d_first, ws.lanes)))
            return rc;
        fs->nk_cap = (int)nk;
    }
    if (!fs->d_loop && (rc = dalloc(&fs->d_loop, 1))) return rc;
    const bool loop = use_graphs(h);
    std::vector<double> lo(nk, a), hi(nk, b);
    CK(cudaMemcpyAsync(fs->d_lo, lo.data(), nk * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(fs->d_hi, hi.data(), nk * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(fs->d_k, k, nk * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    int rounds = 0, nact = 0;
    h->last_rounds = 0;
    h->last_shifts = 0;
    h->last_mixed_rounds = 0;
    if (h->opt.precision == H2_PREC_MIXED) {
        // mixed rounds while the brackets are wider than Delta = 64 u_32 ||A||_inf
        const double delta = guard_delta(h);
        if (loop) {
            int r = 0;
            if ((rc = run_loop(h, (int)nk, std::max(tol, delta), 1, &r))) return rc;
            rounds += r;
            h->last_mixed_rounds += r;
        } else {
            while (true) {
                if ((rc = kth_round(h, (int)nk, std::max(tol, delta), 1, &nact))) return rc;
                if (nact == 0) break;
                ++rounds;
                ++h->last_mixed_rounds;
                if (rounds > 4096) { set_error("h2_kth_eig: no convergence"); return H2_ERR_NUMERICAL; }
            }
        }
        // widen every bracket by Delta and verify it in FP64: nu(lo) < k <= nu(hi);
        // a bracket that fails restarts from the Gershgorin interval
        CK(cudaMemcpyAsync(lo.data(), fs->d_lo, nk * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hi.data(), fs->d_hi, nk * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        std::vector<double> pts;
        for (int64_t i = 0; i < nk; ++i) {
            lo[i] = std::max(a, lo[i] - delta);
            hi[i] = std::min(b, hi[i] + delta);
            pts.push_back(lo[i]);
            pts.push_back(hi[i]);
        }
        std::sort(pts.begin(), pts.end());
        pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
        std::vector<int64_t> cnt(pts.size());
        std::vector<double> mp(pts.size());
        for (size_t b0 = 0; b0 < pts.size(); b0 += ws.lanes) {
            int nb = (int)std::min<size_t>(ws.lanes, pts.size() - b0);
            if ((rc = host_batch(h, pts.data() + b0, nb, 0, cnt.data() + b0, mp.data() + b0))) return rc;
        }
        h->last_shifts += (int64_t)pts.size();
        auto count_at = [&](double x) {
            size_t j = std::lower_bound(pts.begin(), pts.end(), x) - pts.begin();
            return cnt[j];
        };
        for (int64_t i = 0; i < nk; ++i) {
            int64_t cl = (lo[i] == a) ? nu_a : count_at(lo[i]);
            int64_t ch = (hi[i] == b) ? nu_b : count_at(hi[i]);
            if (!(cl < k[i] && k[i] <= ch)) {
                lo[i] = a;
                hi[i] = b;
                ++h->last_bracket_resets;
            }
        }
        CK(cudaMemcpyAsync(fs->d_lo, lo.data(), nk * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(fs->d_hi, hi.data(), nk * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    // FP64 rounds to the requested width (Algorithm 1's stopping rule)
    if (loop) {
        int r = 0;
        if ((rc = run_loop(h, (int)nk, tol, 0, &r))) return rc;
        rounds += r;
    } else {
        while (true) {
            if ((rc = kth_round(h, (int)nk, tol, 0, &nact))) return rc;
            if (nact == 0) break;
            ++rounds;
            if (rounds > 4096) { set_error("h2_kth_eig: bisection did not converge"); return H2_ERR_NUMERICAL; }
        }
    }
    h->last_rounds = rounds;
    CK(cudaMemcpyAsync(lo.data(), fs->d_lo, nk * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hi.data(), fs->d_hi, nk * sizeof(double), cudaMemcpyDeviceToHost, st));
    int err[8] = {0};
    CK(cudaMemcpyAsync(err, ws.d_err, sizeof(err), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err[0]) {
        set_error("h2_kth_eig: " + err_message(err));
        return H2_ERR_NUMERICAL;
    }
    for (int64_t i = 0; i < nk; ++i) {
        out[order[i]] = 0.5 * (lo[i] + hi[i]);
        if (err_bound) err_bound[order[i]] = 0.5 * (hi[i] - lo[i]);
    }
    return H2_OK;
}

void free_workspace(h2_matrix* h) {
    Workspace& ws = h->ws;
    if (ws.graph) cudaGraphExecDestroy(ws.graph);
    if (ws.graph_mixed) cudaGraphExecDestroy(ws.graph_mixed);
    ws.graph = nullptr;
    ws.graph_mixed = nullptr;
    for (auto p : ws.d_slots) cudaFree(p);
    for (auto p : ws.d_dim) cudaFree(p);
    for (auto p : ws.d_rk) cudaFree(p);
    cudaFree(ws.d_scratch); cudaFree(ws.d_merge); cudaFree(ws.d_neg); cudaFree(ws.d_minpiv);
    cudaFree(ws.d_err); cudaFree(ws.d_shifts);
    FactorState* fs = state_of(h);
    if (fs) {
        for (auto& W : fs->lw) {
            for (auto& C : W.colours) {
                cudaFree(C.cl); cudaFree(C.targ); cudaFree(C.targ_slot); cudaFree(C.targ_trans);
                cudaFree(C.ntarg); cudaFree(C.rowblk); cudaFree(C.rowblk_other); cudaFree(C.rowblk_trans);
                cudaFree(C.rowblk_fill);
                cudaFree(C.nrow); cudaFree(C.fillq); cudaFree(C.fillslot); cudaFree(C.nfill); cudaFree(C.pairs);
                cudaFree(C.pairsA); cudaFree(C.pairsB);
            }
            cudaFree(W.d_slot_of); cudaFree(W.d_far_of);
        }
        cudaFree(fs->d_active); cudaFree(fs->d_counts); cudaFree(fs->d_mp); cudaFree(fs->d_stats);
        cudaFree(fs->d_lo); cudaFree(fs->d_hi); cudaFree(fs->d_k); cudaFree(fs->d_nact); cudaFree(fs->d_first);
        cudaFree(fs->d_req); cudaFree(fs->d_gc); cudaFree(fs->d_gmp); cudaFree(fs->d_rr_idx); cudaFree(fs->d_rr_n);
        cudaFree(fs->d_tally);
        cudaFree(fs->d_loop);
        for (auto& e : fs->loop_exec)
            if (e) cudaGraphExecDestroy(e);
        if (fs->side) cudaStreamDestroy(fs->side);
        if (fs->ev_fork) cudaEventDestroy(fs->ev_fork);
        if (fs->ev_join) cudaEventDestroy(fs->ev_join);
        delete fs;
    }
    ws.graph_state = nullptr;
}

}  // namespace h2
