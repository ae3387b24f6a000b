// C ABI entry points (include/h2eig.h): argument checks, error reporting and
// handle lifetime.  All arithmetic runs in the CUDA kernels of h2_build.cu and
// h2_factor.cu.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "h2_internal.h"

namespace h2 {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

void free_device(h2_matrix* h) {
    free_workspace(h);
    for (auto& D : h->lev) {
        cudaFree(D.d_rb); cudaFree(D.d_Q); cudaFree(D.d_C); cudaFree(D.d_slot_a); cudaFree(D.d_slot_b);
        cudaFree(D.d_slot_kind); cudaFree(D.d_slot_far); cudaFree(D.d_off); cudaFree(D.d_color);
        cudaFree(D.d_near_static);
    }
    cudaFree(h->d_points);
}

}  // namespace h2

using namespace h2;

extern "C" {

void h2_default_options(h2_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = H2_PREC_FP64;
    opt->admissibility = H2_ADM_BOX;
    opt->eps_h2 = 1e-10;
    opt->fill_cap = 0;
    opt->sketch_cols = 0;
    opt->seed = 0x5EEDull;
    opt->max_lanes = 64;
    opt->pivot_guard = 1e-3;
    opt->stream = nullptr;
    opt->graphs = 1;
    opt->tc_schur = 0;
    opt->lookahead = 0;
    opt->shifts_per_interval = 16;
}

const char* h2_last_error(void) { return g_last_error.c_str(); }

int h2_build(const double* points, int64_t n, int d, h2_kernel kernel, int leaf, int rank, double eta,
             const h2_options* opt, h2_handle* out) {
    g_last_error.clear();
    if (!points || !out) { set_error("h2_build: null pointer"); return H2_ERR_INVALID_ARG; }
    if (n < 1 || d < 1 || d > 3 || leaf < 2 || rank < 0 || !(eta > 0.0)) {
        set_error("h2_build: need n >= 1, 1 <= d <= 3, leaf >= 2, rank >= 0, eta > 0");
        return H2_ERR_INVALID_ARG;
    }
    if (kernel.kind < 0 || kernel.kind > H2_K_MIN_TEST) { set_error("h2_build: unknown kernel"); return H2_ERR_INVALID_ARG; }
    h2_options o;
    h2_default_options(&o);
    if (opt) o = *opt;
    if (o.max_lanes > 65535) { set_error("h2_build: max_lanes above 65535"); return H2_ERR_INVALID_ARG; }
    if (o.max_lanes <= 0) o.max_lanes = o.hbm_budget > 0 ? 65535 : 64;
    if (!(o.pivot_guard > 0.0)) o.pivot_guard = 1e-3;
    if (!(o.eps_h2 >= 0.0) || o.fill_cap < 0 || o.sketch_cols < 0 ||
        (o.precision != H2_PREC_FP64 && o.precision != H2_PREC_MIXED && o.precision != H2_PREC_FP64_TC) ||
        (o.admissibility != H2_ADM_BOX && o.admissibility != H2_ADM_CENTER && o.admissibility != H2_ADM_WEAK)) {
        set_error("h2_build: invalid options");
        return H2_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < n * d; ++i)
        if (!(points[i] == points[i]) || points[i] > 1e300 || points[i] < -1e300) {
            set_error("h2_build: non-finite point coordinate");
            return H2_ERR_INVALID_ARG;
        }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        set_error("h2_build: no CUDA device");
        return H2_ERR_CUDA;
    }
    h2_matrix* h = new (std::nothrow) h2_matrix();
    if (!h) { set_error("h2_build: host allocation failed"); return H2_ERR_OOM; }
    h->n = n; h->d = d; h->kernel = kernel; h->leaf = leaf; h->rank = rank; h->eta = eta; h->opt = o;
    h->plan_points.assign(points, points + n * d);
    if (o.stream) {
        h->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("h2_build: cudaStreamCreate failed");
            delete h;
            return H2_ERR_CUDA;
        }
        h->own_stream = true;
    }
    h->plan = make_plan(points, n, d, leaf, eta, o.admissibility);
    int rc = build_device(h);
    if (rc == H2_OK && o.hbm_budget > 0) {
        const size_t per = workspace_lane_bytes(h);
        const size_t fit = per > 0 ? o.hbm_budget / per : 0;
        if (fit < 1) {
            set_error("h2_build: one lane's workspace (" + std::to_string(per) + " bytes) exceeds hbm_budget");
            rc = H2_ERR_OOM;
        } else {
            h->opt.max_lanes = (int)std::min<size_t>((size_t)o.max_lanes, fit);
        }
    }
    if (rc == H2_OK) rc = alloc_workspace(h, h->opt.max_lanes);
    if (rc != H2_OK) {
        std::string keep = g_last_error;
        free_device(h);
        if (h->own_stream) cudaStreamDestroy(h->stream);
        delete h;
        g_last_error = keep;
        return rc;
    }
    const auto& lp = h->plan.lev[h->plan.L];
    for (int c = 0; c < lp.nc; ++c)
        for (int e = 0; e < lp.nc; ++e) {
            h->near_pairs += lp.is_near(c, e);
            h->fill_pairs += lp.is_fill(c, e);
        }
    h->plan_points.clear();
    h->plan_points.shrink_to_fit();
    *out = h;
    return H2_OK;
}

void h2_destroy(h2_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_device(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

int h2_inertia(h2_handle h, const double* shifts, int64_t ns, int64_t* counts, double* min_abs_pivot) {
    g_last_error.clear();
    if (!h || (ns > 0 && (!shifts || !counts)) || ns < 0) { set_error("h2_inertia: bad arguments"); return H2_ERR_INVALID_ARG; }
    if (ns == 0) return H2_OK;
    for (int64_t i = 0; i < ns; ++i)
        if (!(shifts[i] == shifts[i])) { set_error("h2_inertia: NaN shift"); return H2_ERR_INVALID_ARG; }
    return run_inertia_host(h, shifts, ns, counts, min_abs_pivot);
}

int h2_inertia_device(h2_handle h, const double* d_shifts, int64_t ns, int64_t* d_counts, double* d_min_abs_pivot) {
    g_last_error.clear();
    if (!h || ns < 0 || (ns > 0 && (!d_shifts || !d_counts))) { set_error("h2_inertia_device: bad arguments"); return H2_ERR_INVALID_ARG; }
    if (ns > h->ws.lanes) { set_error("h2_inertia_device: ns exceeds max_lanes"); return H2_ERR_INVALID_ARG; }
    return run_inertia(h, d_shifts, (int)ns, d_counts, d_min_abs_pivot);
}

int h2_autotune_choice(h2_handle h, int level, int* out) {
    g_last_error.clear();
    if (!h || !out || level < 0 || level > h->plan.L) { set_error("h2_autotune_choice: bad arguments"); return H2_ERR_INVALID_ARG; }
    return tune_choice(h, level, out);
}

int h2_plan_summary(const double* points, int64_t n, int d, int leaf, double eta, int rule,
                    int64_t* perm, int* levels, int64_t* per_level, int* colours) {
    g_last_error.clear();
    if (!points || !levels || n < 1 || d < 1 || d > 3 || leaf < 2 || !(eta > 0.0) ||
        (rule != H2_ADM_BOX && rule != H2_ADM_CENTER && rule != H2_ADM_WEAK)) {
        set_error("h2_plan_summary: bad arguments");
        return H2_ERR_INVALID_ARG;
    }
    Plan P = make_plan(points, n, d, leaf, eta, rule);
    if (P.L + 1 > 64) { set_error("h2_plan_summary: more than 64 levels"); return H2_ERR_INVALID_ARG; }
    *levels = P.L + 1;
    if (perm)
        for (int64_t i = 0; i < n; ++i) perm[i] = P.perm[i];
    int64_t pos = 0;
    for (int l = 0; l <= P.L; ++l) {
        const LevelPlan& lp = P.lev[l];
        if (per_level) {
            int64_t nn = 0, nf = 0, nfar = 0;
            for (int c = 0; c < lp.nc; ++c)
                for (int e = 0; e < lp.nc; ++e) {
                    nn += lp.is_near(c, e);
                    nf += lp.is_fill(c, e);
                    nfar += lp.is_far(c, e);
                }
            per_level[5 * l] = lp.nc;
            per_level[5 * l + 1] = nn;
            per_level[5 * l + 2] = nf;
            per_level[5 * l + 3] = nfar;
            per_level[5 * l + 4] = (int64_t)lp.color_lists.size();
        }
        if (colours)
            for (int c = 0; c < lp.nc; ++c) colours[pos + c] = lp.color[c];
        pos += lp.nc;
    }
    return H2_OK;
}

int h2_group_create(const h2_handle* hs, int nh, h2_group* out) {
    g_last_error.clear();
    if (!hs || !out || nh < 1) { set_error("h2_group_create: bad arguments"); return H2_ERR_INVALID_ARG; }
    for (int i = 0; i < nh; ++i)
        if (!hs[i]) { set_error("h2_group_create: null handle"); return H2_ERR_INVALID_ARG; }
    return group_create(hs, nh, out);
}

int h2_group_inertia_device(h2_group g, const double* d_shifts, const int* ns, int64_t* d_counts,
                            double* d_min_abs_pivot) {
    g_last_error.clear();
    if (!g || !d_shifts || !ns || !d_counts) { set_error("h2_group_inertia_device: bad arguments"); return H2_ERR_INVALID_ARG; }
    return group_inertia(g, d_shifts, ns, d_counts, d_min_abs_pivot);
}

int h2_group_launches(h2_group g) { return g ? group_launches(g) : -1; }

void h2_group_destroy(h2_group g) { group_destroy(g); }

int h2_kth_eig(h2_handle h, const int64_t* k, int64_t nk, double tol, double* out, double* err_bound) {
    g_last_error.clear();
    if (!h || nk < 0 || (nk > 0 && (!k || !out)) || !(tol > 0.0)) { set_error("h2_kth_eig: bad arguments"); return H2_ERR_INVALID_ARG; }
    for (int64_t i = 0; i < nk; ++i)
        if (k[i] < 1 || k[i] > h->n) { set_error("h2_kth_eig: k out of 1..n"); return H2_ERR_INVALID_ARG; }
    if (nk == 0) return H2_OK;
    return run_kth(h, k, nk, tol, out, err_bound, nullptr);
}

int h2_kth_eig_in(h2_handle h, const int64_t* k, int64_t nk, double lo, double hi, double tol, double* out,
                  double* err_bound) {
    g_last_error.clear();
    if (!h || nk < 0 || (nk > 0 && (!k || !out)) || !(tol > 0.0) || !(lo < hi)) {
        set_error("h2_kth_eig_in: bad arguments");
        return H2_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < nk; ++i)
        if (k[i] < 1 || k[i] > h->n) { set_error("h2_kth_eig_in: k out of 1..n"); return H2_ERR_INVALID_ARG; }
    if (nk == 0) return H2_OK;
    const double iv[2] = {lo, hi};
    return run_kth(h, k, nk, tol, out, err_bound, iv);
}

int h2_info(h2_handle h, h2_stats* s) {
    if (!h || !s) { set_error("h2_info: null pointer"); return H2_ERR_INVALID_ARG; }
    std::memset(s, 0, sizeof(*s));
    s->n = h->n;
    s->levels = h->plan.L + 1;
    s->leaves = h->plan.lev[h->plan.L].nc;
    s->max_rank = h->max_rank;
    s->near_pairs = h->near_pairs;
    s->fill_pairs = h->fill_pairs;
    s->norm_inf = h->norm_inf;
    s->gershgorin_lo = h->glo;
    s->gershgorin_hi = h->ghi;
    s->trunc_tol = h->tol;
    s->workspace_bytes = (int64_t)h->ws.bytes;
    s->lanes = h->ws.lanes;
    s->kernels_per_batch = h->kernels_per_batch;
    s->last_rounds = h->last_rounds;
    s->last_shifts = h->last_shifts;
    s->last_mixed_rounds = h->last_mixed_rounds;
    int64_t checked = 0, reruns = 0;
    int rc = guard_tally(h, &checked, &reruns);
    if (rc) return rc;
    s->guard_reruns = reruns;
    s->guard_checked = checked;
    s->bracket_resets = h->last_bracket_resets;
    for (const auto& D : h->lev)
        for (double r : D.resid) {
            s->cap_bound += r > h->tol ? 1 : 0;
            s->max_residual = std::max(s->max_residual, r);
        }
    return H2_OK;
}

int h2_export(h2_handle h, h2_export_buf* buf) {
    g_last_error.clear();
    if (!h || !buf) { set_error("h2_export: null pointer"); return H2_ERR_INVALID_ARG; }
    return run_export(h, buf);
}

int h2_compression_error(h2_handle h, int iters, double* err2, double* norm2) {
    g_last_error.clear();
    if (!h || !err2 || !norm2 || iters < 1) { set_error("h2_compression_error: bad arguments"); return H2_ERR_INVALID_ARG; }
    return run_compression_error(h, iters, err2, norm2);
}

int h2_profile_batch(h2_handle h, const double* d_shifts, int64_t ns, int64_t* d_counts, double* ms,
                     int64_t* launches, double* flops, double* bytes) {
    g_last_error.clear();
    if (!h || !d_shifts || !d_counts || !ms || !launches || !flops || !bytes) {
        set_error("h2_profile_batch: null pointer");
        return H2_ERR_INVALID_ARG;
    }
    return run_profile(h, d_shifts, (int)ns, d_counts, ms, launches, flops, bytes);
}

int h2_status(h2_handle h, int64_t* info) {
    g_last_error.clear();
    if (!h || !info) { set_error("h2_status: null pointer"); return H2_ERR_INVALID_ARG; }
    return run_status(h, info);
}

void h2_heartbeat(uint32_t* out) {
    if (out) heartbeat_read(out);
}

int h2_tree_perm(h2_handle h, int64_t* perm) {
    if (!h || !perm) { set_error("h2_tree_perm: null pointer"); return H2_ERR_INVALID_ARG; }
    std::memcpy(perm, h->plan.perm.data(), h->n * sizeof(int64_t));
    return H2_OK;
}

int h2_level_ranks(h2_handle h, int level, int* ranks) {
    if (!h || !ranks || level < 0 || level > h->plan.L) { set_error("h2_level_ranks: bad arguments"); return H2_ERR_INVALID_ARG; }
    const auto& D = h->lev[level];
    std::memcpy(ranks, D.rb.data(), D.nc * sizeof(int));
    return H2_OK;
}

}  // extern "C"
