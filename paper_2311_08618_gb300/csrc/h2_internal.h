// Internal host-side structures of the h2eig library (not part of the C ABI).
//
// A handle owns: the cluster tree and block structure (host planner), the
// resident H^2 representation on the device (bases, couplings, transformed
// leaf near blocks), and the per-batch factorization workspace.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/h2eig.h"

namespace h2 {

// ---------------------------------------------------------------- planner --
struct LevelPlan {
    int nc = 0;                          // clusters at this level
    std::vector<int64_t> off;            // nc + 1 ranges in tree order
    std::vector<uint8_t> near, fill, far;// nc * nc flags (row-major)
    std::vector<int> color;              // distance-2 colour of each cluster
    std::vector<std::vector<int>> color_lists;  // clusters of each colour, ascending
    bool is_near(int c, int d) const { return near[(size_t)c * nc + d] != 0; }
    bool is_fill(int c, int d) const { return fill[(size_t)c * nc + d] != 0; }
    bool is_far(int c, int d) const { return far[(size_t)c * nc + d] != 0; }
};

struct Plan {
    int64_t n = 0;
    int d = 0;
    int L = 0;                           // leaf level (root = 0)
    std::vector<int64_t> perm;           // tree position -> input index
    std::vector<LevelPlan> lev;          // 0..L
};

// Builds the tree, the top-down block tree, the fill-in closure and the
// colouring (same readings as the CPU oracle; independent implementation).
Plan make_plan(const double* pts, int64_t n, int d, int leaf, double eta, int rule);

// ------------------------------------------------------- device resident --
// Work-list entry of one Schur update S_ab -= W_a Y_b^T of one elimination.
struct SchurPair {
    int elim;      // index of the eliminated cluster within its colour list
    int ta, tb;    // target indices of a and b within that cluster's target list
    int slot;      // slot of the stored block (max(a,b), min(a,b))
    int trans;     // 1 if the stored block is (b, a): update its transpose
    int a, b;      // cluster ids
};

// Per-level device data and work lists.
struct LevelDev {
    int nc = 0;
    int dmax = 0;          // padded block dimension in the factorization
    int dq = 0;            // padded dimension of the basis / transfer matrices
    int rbmax = 0;         // max build rank at this level
    int skcap = 0;         // max skeleton size after recompression
    int nslots = 0;        // stored (c >= d) near-or-fill blocks
    int nfar = 0;          // stored (c > d) far couplings
    std::vector<int> slot_of;      // nc*nc -> slot id (for c >= d), -1 otherwise
    std::vector<int> far_of;       // nc*nc -> coupling id (for c > d), -1 otherwise
    std::vector<int> slot_a, slot_b;   // slot -> (c, d)
    std::vector<int> rb;           // build rank per cluster
    std::vector<double> resid;     // Frobenius norm of the sketch remainder left out by the truncation
    // device arrays
    int* d_rb = nullptr;           // [nc]
    double* d_Q = nullptr;         // [nc][dq][dq] bases (leaf) / transfers (upper)
    double* d_C = nullptr;         // [nfar][rbmax][rbmax] couplings
    int* d_slot_a = nullptr;       // [nslots]
    int* d_slot_b = nullptr;       // [nslots]
    int* d_slot_kind = nullptr;    // [nslots] 0 near, 1 fill
    int* d_slot_far = nullptr;     // [nslots] coupling id for fill slots, else -1
    // per-colour work lists (device copies), built at build time
    struct Colour {
        int ncl = 0;                    // clusters in the colour
        int ntarg_max = 0;
        int npairs = 0;
        int* d_cl = nullptr;            // [ncl] cluster ids
        int* d_targ = nullptr;          // [ncl][ntarg_max] target clusters (-1 pad), [0] = self
        int* d_targ_slot = nullptr;     // [ncl][ntarg_max] slot of (t, p) block
        int* d_targ_trans = nullptr;    // [ncl][ntarg_max] 1 if stored as (p, t)
        int* d_ntarg = nullptr;         // [ncl]
        int* d_rowblk = nullptr;        // [ncl][nrow_max] slots of all blocks in row p
        int* d_rowblk_other = nullptr;  // [ncl][nrow_max] the other cluster x of block (p,x)
        int* d_nrow = nullptr;          // [ncl]
        int nrow_max = 0;
        int* d_fillq = nullptr;         // [ncl][nfill_max] fill neighbours q (ascending)
        int* d_fillslot = nullptr;      // [ncl][nfill_max]
        int* d_nfill = nullptr;         // [ncl]
        int nfill_max = 0;
        SchurPair* d_pairs = nullptr;   // [npairs]
    };
    std::vector<Colour> colours;
    int estride = 1;               // columns of the expanded basis E (build only)
    int64_t* d_off = nullptr;      // [nc + 1] cluster ranges in tree order
    int* d_color = nullptr;        // [nc] colour of each cluster
    double* d_near_static = nullptr; // leaf only: [nslots][dmax][dmax] Q_c^T A_cd Q_d
};

struct Workspace {
    int lanes = 0;
    std::vector<double*> d_slots;  // per level [nslots][lanes][dmax*dmax]
    std::vector<int*> d_dim;       // per level [nc][lanes]
    std::vector<int*> d_rk;        // per level [nc][lanes]
    double* d_scratch = nullptr;   // factor-step scratch (two halves with the lookahead schedule)
    size_t scratch_half = 0;       // doubles of one half
    size_t scratch_per_elim = 0;   // doubles per (cluster, lane)
    double* d_merge = nullptr;     // merge scratch
    size_t merge_doubles = 0;
    unsigned long long* d_neg = nullptr;   // [lanes]
    unsigned long long* d_minpiv = nullptr;// [lanes] bit pattern of a non-negative double
    int* d_err = nullptr;          // error flags
    double* d_shifts = nullptr;    // [lanes]
    size_t bytes = 0;
    cudaGraphExec_t graph = nullptr;        // FP64 batch
    cudaGraphExec_t graph_mixed = nullptr;  // mixed-precision batch
    void* graph_state = nullptr;   // factorization work lists (h2_factor.cu)
};

}  // namespace h2

struct h2_matrix {
    h2::Plan plan;
    std::vector<h2::LevelDev> lev;
    h2::Workspace ws;
    int64_t n = 0;
    int d = 0;
    h2_kernel kernel{};
    int leaf = 0, rank = 0;
    double eta = 1.0;
    h2_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double norm_inf = 0, glo = 0, ghi = 0, tol = 0;
    int max_rank = 0;
    int64_t near_pairs = 0, fill_pairs = 0;
    double* d_points = nullptr;    // [n][3] tree order (padded to 3 coordinates)
    std::vector<double> plan_points;  // host copy of the input points (n x d)
    int mmax = 0;                  // largest leaf
    int fill_cap_eff = 0;          // skeleton cap after recompression
    // autotuned kernel choices per level (0 / -1: the default rules)
    std::vector<int> tune_ldl;       // k_ldl threads per CTA (128 or 256)
    std::vector<int> tune_recomp;    // 1: clustered recompression, 0: one CTA
    int last_rounds = 0;           // bisection rounds of the last h2_kth_eig
    int64_t last_shifts = 0;       // shifts evaluated by the last h2_kth_eig
    int kernels_per_batch = 0;     // launches in one batch (graph nodes)
    int last_mixed_rounds = 0;     // mixed rounds of the last h2_kth_eig
    int64_t last_bracket_resets = 0;  // brackets that failed the FP64 verification
};

namespace h2 {
void set_error(const std::string& msg);
int build_device(h2_matrix* h);                         // construction kernels
int alloc_workspace(h2_matrix* h, int lanes);
size_t workspace_lane_bytes(h2_matrix* h);      // device bytes per lane
int run_inertia(h2_matrix* h, const double* d_shifts, int ns, int64_t* d_counts,
                double* d_minpiv);                    // enqueue one batch
int run_inertia_host(h2_matrix* h, const double* shifts, int64_t ns, int64_t* counts,
                     double* minpiv);
int run_profile(h2_matrix* h, const double* d_shifts, int ns, int64_t* d_counts, double* ms,
                int64_t* launches, double* flops, double* bytes);
int run_kth(h2_matrix* h, const int64_t* k, int64_t nk, double tol, double* out,
            double* err_bound, const double* interval);   // interval: nullable [lo, hi]
void free_workspace(h2_matrix* h);
int run_status(h2_matrix* h, int64_t* info);
int tune_choice(h2_matrix* h, int level, int* out);
int group_create(h2_matrix* const* hs, int nh, h2_group_set** out);
int group_inertia(h2_group_set* g, const double* d_shifts, const int* ns, int64_t* d_counts, double* d_minpiv);
int group_launches(const h2_group_set* g);
void group_destroy(h2_group_set* g);
void heartbeat_read(unsigned int* out);
void free_device(h2_matrix* h);
int run_export(h2_matrix* h, h2_export_buf* buf);
int guard_tally(h2_matrix* h, int64_t* checked, int64_t* rerun);   // mixed guard totals
int run_compression_error(h2_matrix* h, int iters, double* err2, double* norm2);
}  // namespace h2
