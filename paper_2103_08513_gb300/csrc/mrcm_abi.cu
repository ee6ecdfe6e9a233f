// extern "C" entry points of libmrcm (declared in include/mrcm.h).
#include <cuda_runtime.h>

#include <map>
#include <tuple>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>
#include <algorithm>
#include <cstring>
#include <new>

#include "mrcm_internal.h"

using mrcm::Tables;

namespace {

thread_local std::string g_setup_err;   // message of the last failed mrcm_setup on this thread

mrcm_status fail(mrcm_handle* h, mrcm_status st, const std::string& msg) {
    if (h) h->err = msg;
    return st;
}

mrcm_status cuda_fail(mrcm_handle* h, cudaError_t e, const char* where) {
    return fail(h, MRCM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
    size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)dst, bytes);
    if (e != cudaSuccess) return e;
    if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

void load_tune_cache(mrcm_handle* h);

void free_device(mrcm::DeviceTables& d) {
    void* ptrs[] = {d.subs, d.faces, d.Ilist, d.class_list, d.solve_list, d.rowptr, d.colidx, d.src_lo, d.src_hi, d.rhs_src_lo,
                    d.rhs_src_hi, d.fronts, d.front_maps, d.front_inv, d.front_dofs, d.level_ids, d.pp_subs};
    for (void* p : ptrs) if (p) cudaFree(p);
    d = mrcm::DeviceTables();
}

mrcm_status ensure_device(mrcm_handle* h, void* stream) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
    if (h->d.ready) {
        if (dev != h->d.device) return fail(h, MRCM_ERR_STATE, "handle was set up on another device");
        return MRCM_OK;
    }
    // make sure nothing queued on the caller's stream still reads the tables we replace
    if (stream) cudaStreamSynchronize((cudaStream_t)stream);
    const Tables& t = h->t;
    mrcm::DeviceTables& d = h->d;
    std::vector<int> lvl;
    d.level_off.assign(t.levels.size() + 1, 0);
    for (size_t k = 0; k < t.levels.size(); ++k) {
        d.level_off[k] = (int)lvl.size();
        lvl.insert(lvl.end(), t.levels[k].begin(), t.levels[k].end());
    }
    d.level_off[t.levels.size()] = (int)lvl.size();
#define UP(dst, src) do { e = upload(&d.dst, src); if (e != cudaSuccess) { free_device(d); return cuda_fail(h, e, "table upload"); } } while (0)
    UP(subs, t.subs);
    UP(faces, t.faces);
    UP(Ilist, t.Ilist);
    UP(class_list, t.class_list);
    UP(solve_list, t.solve_list);
    for (int q = 0; q < 4; ++q) d.class_off[q] = t.class_off[q];
    UP(rowptr, t.rowptr);
    UP(colidx, t.colidx);
    UP(src_lo, t.src_lo);
    UP(src_hi, t.src_hi);
    UP(rhs_src_lo, t.rhs_src_lo);
    UP(rhs_src_hi, t.rhs_src_hi);
    UP(fronts, t.fronts);
    UP(front_maps, t.front_maps);
    UP(front_inv, t.front_inv);
    UP(front_dofs, t.front_dofs);
    UP(level_ids, lvl);
    if (!t.pp_subs.empty()) UP(pp_subs, t.pp_subs);
#undef UP
    int rc = mrcm::configure_local(t, d);
    if (!rc) rc = mrcm::configure_interface(t, d);
    if (!rc) rc = mrcm::configure_reconstruct(t);
    if (rc) { free_device(d); return cuda_fail(h, (cudaError_t)rc, "kernel configuration"); }
    load_tune_cache(h);
    d.device = dev;
    d.ready = true;
    return MRCM_OK;
}

std::string tune_key(const mrcm_handle* h) {
    const Tables& t = h->t;
    char buf[256];
    snprintf(buf, sizeof(buf), "n%lld_s%d_b%d_m%d_N%d_r%lld_p%d", t.n_cells, (int)t.subs.size(), t.max_b, t.max_m,
             t.max_N, t.total_rhs, t.cfg.precision);
    return buf;
}

// Tune cache: text lines "key solve_variant sweep_variant factor_variant factor_mid_variant
// [sweeps_separate]" (the last field is optional: 0 when absent).
void load_tune_cache(mrcm_handle* h) {
    if (h->t.tune_cache.empty()) return;
    FILE* fp = fopen(h->t.tune_cache.c_str(), "r");
    if (!fp) return;
    char line[512], key[256];
    const std::string want = tune_key(h);
    while (fgets(line, sizeof(line), fp)) {
        int v0, v1, v2, v3, v4 = 0;
        const int n = sscanf(line, "%255s %d %d %d %d %d", key, &v0, &v1, &v2, &v3, &v4);
        if (n < 5) continue;
        if (want == key && v0 >= 0 && v0 < mrcm::num_solve_variants() && v1 >= 0 && v1 < mrcm::num_solve_variants() &&
            v2 >= 0 && v2 < mrcm::kNumFactorVariants && (v3 == 0 || v3 == 1) && (v4 == 0 || v4 == 1)) {
            h->d.solve_variant = v0;
            h->d.sweep_variant = v1;
            h->d.factor_variant = v2;
            h->d.factor_mid_variant = v3;
            h->d.sweeps_separate = v4;
        }
    }
    fclose(fp);
}

void store_tune_cache(mrcm_handle* h) {
    if (h->t.tune_cache.empty()) return;
    std::vector<std::string> keep;
    const std::string want = tune_key(h);
    if (FILE* fp = fopen(h->t.tune_cache.c_str(), "r")) {
        char line[512], key[256];
        while (fgets(line, sizeof(line), fp)) {
            int v[5] = {0, 0, 0, 0, 0};
            const int n = sscanf(line, "%255s %d %d %d %d %d", key, &v[0], &v[1], &v[2], &v[3], &v[4]);
            if (n >= 5 && want != key)
                keep.push_back(std::string(key) + " " + std::to_string(v[0]) + " " + std::to_string(v[1]) + " " +
                               std::to_string(v[2]) + " " + std::to_string(v[3]) + " " + std::to_string(v[4]));
        }
        fclose(fp);
    }
    if (FILE* fp = fopen(h->t.tune_cache.c_str(), "w")) {
        for (auto& line : keep) fprintf(fp, "%s\n", line.c_str());
        fprintf(fp, "%s %d %d %d %d %d\n", want.c_str(), h->d.solve_variant, h->d.sweep_variant, h->d.factor_variant,
                h->d.factor_mid_variant, h->d.sweeps_separate);
        fclose(fp);
    }
}

void drop_graph(mrcm_handle* h) {
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->graph_exec = nullptr;
    h->graph = nullptr;
}

mrcm_status check_ws(mrcm_handle* h, const void* ws) {
    if (!ws) return fail(h, MRCM_ERR_INVALID_ARG, "workspace is NULL");
    if (((uintptr_t)ws & 255u) != 0) return fail(h, MRCM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    return MRCM_OK;
}

mrcm_status after_launch(mrcm_handle* h, int rc, const char* where) {
    if (rc != 0) return cuda_fail(h, (cudaError_t)rc, where);
    return MRCM_OK;
}

}  // namespace

extern "C" {

mrcm_status mrcm_setup(const mrcm_config* cfg, mrcm_handle** out) {
    if (!out) return MRCM_ERR_INVALID_ARG;
    *out = nullptr;
    mrcm_handle* h = new (std::nothrow) mrcm_handle();
    if (!h) return MRCM_ERR_OOM;
    mrcm_status st = mrcm::build_tables(cfg, h->t, h->err);
    const Tables& t = h->t;
    if (st == MRCM_OK) {
        for (const auto& s : t.subs) {
            if (s.nI > mrcm::kMaxI) { st = MRCM_ERR_NOT_IMPLEMENTED; h->err = "too many basis functions on one subdomain"; break; }
            if (s.N > 4096) { st = MRCM_ERR_NOT_IMPLEMENTED; h->err = "subdomain larger than 4096 cells"; break; }
        }
    }
    const int mpad = (t.max_m + 3) & ~3;
    size_t solve_smem = 0;
    for (const auto& sb : t.subs)
        solve_smem = std::max(solve_smem, t.cfg.precision == MRCM_FP64 ? mrcm::solve_smem_layout<double>(sb.b, mpad, sb.N).total
                                                                          : mrcm::solve_smem_layout<float>(sb.b, mpad, sb.N).total);
    if (st == MRCM_OK && solve_smem + 16 > 227 * 1024) {
        st = MRCM_ERR_NOT_IMPLEMENTED;
        h->err = "slab block and right-hand-side count exceed shared memory";
    }
    if (st != MRCM_OK) {
        g_setup_err = h->err;
        delete h;
        return st;
    }
    mrcm::compute_layout(h->t, h->lay);
    *out = h;
    return MRCM_OK;
}

mrcm_status mrcm_query_workspace(const mrcm_handle* h, size_t* ws_bytes, size_t* n_iface) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    if (ws_bytes) *ws_bytes = h->lay.total;
    if (n_iface) *n_iface = (size_t)2 * h->t.NV;
    return MRCM_OK;
}

mrcm_status mrcm_query_sizes(const mrcm_handle* h, mrcm_sizes* o) {
    if (!h || !o) return MRCM_ERR_INVALID_ARG;
    const Tables& t = h->t;
    std::memset(o, 0, sizeof(*o));
    o->n_cells = t.n_cells;
    o->n_sub = (int)t.subs.size();
    o->n_basis = t.NV;
    o->n_faces = (long long)t.faces.size();
    o->max_rhs = t.max_m;
    o->total_rhs = t.total_rhs;
    o->nnz_interface = (long long)t.colidx.size();
    o->n_fronts = (int)t.fronts.size();
    o->max_front = t.max_front;
    o->front_flops = t.front_flops;
    o->local_factor_flops = t.local_factor_flops;
    o->local_solve_flops = t.local_solve_flops;
    o->max_block = t.max_b;
    o->mbf_entries = t.total_x;
    o->ldl_flops = t.ldl_flops;
    o->ldl_update_flops = t.ldl_update_flops;
    o->ldl_update_tensor_flops = t.ldl_update_tensor_flops;
    o->n_waves = t.n_waves;
    o->max_front_ne = 0;
    o->max_front_nb = 0;
    for (const auto& f : t.fronts) {
        o->max_front_ne = std::max(o->max_front_ne, f.ne);
        o->max_front_nb = std::max(o->max_front_nb, f.nb);
    }
    return MRCM_OK;
}

mrcm_status mrcm_query_local_ldl(const mrcm_handle* h, double* factor_flops, double* solve_flops) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    const Tables& t = h->t;
    if (t.max_N > 4096) return fail(const_cast<mrcm_handle*>(h), MRCM_ERR_NOT_IMPLEMENTED, "subdomain above 4096 cells");
    std::map<std::tuple<int, int, int>, std::pair<double, long long>> cache;
    double ff = 0.0, sf = 0.0;
    for (const auto& s : t.subs) {
        const auto key = std::make_tuple(s.sz[0], s.sz[1], s.sz[2]);
        auto it = cache.find(key);
        if (it == cache.end()) {
            double fl;
            long long nz;
            mrcm::min_degree_cost(s.sz[0], s.sz[1], s.sz[2], &fl, &nz);
            it = cache.emplace(key, std::make_pair(fl, nz)).first;
        }
        ff += it->second.first;
        sf += 4.0 * (double)it->second.second * s.m;
    }
    if (factor_flops) *factor_flops = ff;
    if (solve_flops) *solve_flops = sf;
    return MRCM_OK;
}

mrcm_status mrcm_query_basis(const mrcm_handle* h, int i, int* axis, int* lo, int* hi, int* nf) {
    if (!h || i < 0 || i >= h->t.NV) return MRCM_ERR_INVALID_ARG;
    if (axis) *axis = h->t.b_axis[i];
    if (lo) *lo = h->t.b_lo[i];
    if (hi) *hi = h->t.b_hi[i];
    if (nf) *nf = h->t.b_nfaces[i];
    return MRCM_OK;
}

mrcm_status mrcm_factor_local(mrcm_handle* h, const double* K, void* ws, size_t ws_bytes, void* stream) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    if (!K) return fail(h, MRCM_ERR_INVALID_ARG, "K is NULL");
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    if (ws_bytes < h->lay.total) return fail(h, MRCM_ERR_OOM, "workspace smaller than mrcm_query_workspace");
    if ((st = ensure_device(h, stream)) != MRCM_OK) return st;
    h->K = K;
    int rc = mrcm::launch_factor(h->t, h->d, h->lay, (char*)ws, K, h->t.cfg.precision, stream, h->prof);
    if ((st = after_launch(h, rc, "mrcm_factor_local")) != MRCM_OK) return st;
    h->stage = 1;
    return MRCM_OK;
}

mrcm_status mrcm_solve_mbf(mrcm_handle* h, const double* f, void* ws, void* stream) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    if (!f) return fail(h, MRCM_ERR_INVALID_ARG, "f is NULL");
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    if (h->stage < 1) return fail(h, MRCM_ERR_STATE, "mrcm_factor_local must run first");
    if (h->t.cfg.precision == MRCM_LEARNED_PCG)
        return fail(h, MRCM_ERR_INVALID_ARG, "the learned form solves its MBFs with mrcm_solve_mbf_learned");
    h->f = f;
    int sweeps = h->t.cfg.precision == MRCM_FP64 ? 0 : h->t.cfg.ir_max_sweeps;
    double tol = h->t.cfg.ir_tol > 0 ? h->t.cfg.ir_tol : 1e-14;
    int rc = mrcm::launch_solve_mbf(h->t, h->d, h->lay, (char*)ws, f, h->t.cfg.precision, sweeps, tol, stream, h->prof);
    if ((st = after_launch(h, rc, "mrcm_solve_mbf")) != MRCM_OK) return st;
    h->stage = 2;
    return MRCM_OK;
}

mrcm_status mrcm_assemble_interface(mrcm_handle* h, void* ws, void* stream) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    if (h->stage < 2) return fail(h, MRCM_ERR_STATE, "mrcm_solve_mbf must run first");
    int rc = mrcm::launch_assemble_interface(h->t, h->d, h->lay, (char*)ws, stream, h->prof);
    if ((st = after_launch(h, rc, "mrcm_assemble_interface")) != MRCM_OK) return st;
    h->stage = 3;
    return MRCM_OK;
}

mrcm_status mrcm_solve_interface(mrcm_handle* h, double* X, void* ws, void* stream) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    if (!X && h->t.NV > 0) return fail(h, MRCM_ERR_INVALID_ARG, "X is NULL");
    if (h->stage < 3) return fail(h, MRCM_ERR_STATE, "mrcm_assemble_interface must run first");
    int rc = mrcm::launch_solve_interface(h->t, h->d, h->lay, (char*)ws, X, stream, h->prof);
    if ((st = after_launch(h, rc, "mrcm_solve_interface")) != MRCM_OK) return st;
    h->stage = 4;
    return MRCM_OK;
}

mrcm_status mrcm_reconstruct(mrcm_handle* h, const double* X, double* p, double* u, double* mres, void* ws,
                             void* stream) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    if (!p || !u || (!X && h->t.NV > 0)) return fail(h, MRCM_ERR_INVALID_ARG, "X, p and u must be non-NULL");
    if (h->stage < 4) return fail(h, MRCM_ERR_STATE, "mrcm_solve_interface must run first");
    int rc = mrcm::launch_reconstruct(h->t, h->d, h->lay, (char*)ws, X, p, u, mres, h->K, h->f, stream, h->prof);
    return after_launch(h, rc, "mrcm_reconstruct");
}

mrcm_status mrcm_postprocess_velocity(mrcm_handle* h, const double* u, double* u_out, double* mres, void* ws,
                                      void* stream) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    if (!u || !u_out) return fail(h, MRCM_ERR_INVALID_ARG, "u and u_out must be non-NULL");
    const size_t ub = (size_t)6 * h->t.n_cells * sizeof(double);
    const char* a = (const char*)u;
    const char* b = (const char*)u_out;
    if (a < b + ub && b < a + ub) return fail(h, MRCM_ERR_INVALID_ARG, "u and u_out overlap");
    if (h->stage < 4) return fail(h, MRCM_ERR_STATE, "the multiscale solve must run first");
    if (!h->t.pp_ok) return fail(h, MRCM_ERR_NOT_IMPLEMENTED, "a slab block too large for the FP64 post-processing factor");
    const int precision = h->t.cfg.precision;
    const int sweeps = 3;                // FP64 refinement steps of the FP64 Neumann solves
    const double tol = h->t.cfg.ir_tol > 0 ? h->t.cfg.ir_tol : 1e-14;
    int rc = mrcm::launch_postprocess(h->t, h->d, h->lay, (char*)ws, u, u_out, mres, h->f, precision, sweeps, tol,
                                      stream, h->prof);
    h->stage = 0;                        // coefficients, factors and MBF columns are overwritten
    return after_launch(h, rc, "mrcm_postprocess_velocity");
}

mrcm_status mrcm_read_status(mrcm_handle* h, void* ws, int* not_spd, int* unconverged, int* zero_piv,
                             int* sweeps) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    int w[mrcm::ST_COUNT];
    cudaError_t e = cudaMemcpy(w, (char*)ws + h->lay.status, sizeof(w), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "mrcm_read_status");
    if (not_spd) *not_spd = w[mrcm::ST_NOT_SPD];
    if (unconverged) *unconverged = w[mrcm::ST_UNCONVERGED];
    if (zero_piv) *zero_piv = w[mrcm::ST_ZERO_PIVOT];
    if (sweeps) *sweeps = w[mrcm::ST_SWEEPS];
    if (w[mrcm::ST_NOT_SPD]) return fail(h, MRCM_ERR_NOT_SPD, "non-positive local block pivot");
    if (w[mrcm::ST_ZERO_PIVOT]) return fail(h, MRCM_ERR_SINGULAR_INTERFACE, "zero pivot in the interface factorisation");
    if (w[mrcm::ST_UNCONVERGED]) return fail(h, MRCM_ERR_NO_CONVERGENCE, "iterative refinement did not converge");
    return MRCM_OK;
}

mrcm_status mrcm_read_fallback(mrcm_handle* h, void* ws, int* fallback_subdomains, int* not_recovered) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    int w[mrcm::ST_COUNT];
    cudaError_t e = cudaMemcpy(w, (char*)ws + h->lay.status, sizeof(w), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "mrcm_read_fallback");
    if (fallback_subdomains) *fallback_subdomains = w[mrcm::ST_FB_TOTAL];
    if (not_recovered) *not_recovered = w[mrcm::ST_FB_LOST];
    return MRCM_OK;
}

mrcm_status mrcm_read_work(mrcm_handle* h, void* ws, long long* swept) {
    if (!h || !swept) return MRCM_ERR_INVALID_ARG;
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    unsigned long long v = 0;
    cudaError_t e = cudaMemcpy(&v, (char*)ws + h->lay.status + mrcm::ST_SWEPT * sizeof(int), sizeof(v),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "mrcm_read_work");
    *swept = (long long)v;
    return MRCM_OK;
}

mrcm_status mrcm_export(mrcm_handle* h, void* ws, int what, int sub, void* dst, size_t bytes) {
    if (!h || !dst) return MRCM_ERR_INVALID_ARG;
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    const Tables& t = h->t;
    const char* w = (const char*)ws;
    cudaError_t e = cudaSuccess;
    size_t need = 0;
    const void* src = nullptr;
    switch (what) {
        case 0: need = t.colidx.size() * sizeof(double); src = w + h->lay.csr_val; break;
        case 1: need = (size_t)2 * t.NV * sizeof(double); src = w + h->lay.b_int; break;
        case 2:
            need = t.rowptr.size() * sizeof(int);
            if (bytes < need) return fail(h, MRCM_ERR_INVALID_ARG, "export buffer too small");
            std::memcpy(dst, t.rowptr.data(), need);
            return MRCM_OK;
        case 3:
            need = t.colidx.size() * sizeof(int);
            if (bytes < need) return fail(h, MRCM_ERR_INVALID_ARG, "export buffer too small");
            std::memcpy(dst, t.colidx.data(), need);
            return MRCM_OK;
        case 4: {
            if (sub < 0 || sub >= (int)t.subs.size()) return fail(h, MRCM_ERR_INVALID_ARG, "bad subdomain");
            const mrcm::SubInfo& s = t.subs[sub];
            need = (size_t)s.m * s.N * sizeof(double);
            if (bytes < need) return fail(h, MRCM_ERR_INVALID_ARG, "export buffer too small");
            std::vector<double> tmp((size_t)s.m * s.N);
            e = cudaMemcpy(tmp.data(), w + h->lay.X + s.x_off * sizeof(double), need, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(h, e, "mrcm_export");
            // slab order -> lexicographic order (x fastest) inside the subdomain box
            double* out = (double*)dst;
            for (int c = 0; c < s.N; ++c) {
                int sl = c / s.b, r = c % s.b, v = r / s.su, uu = r % s.su;
                int lc[3];
                lc[s.sa] = sl; lc[s.ua] = uu; lc[s.va] = v;
                int lex = lc[0] + s.sz[0] * (lc[1] + s.sz[1] * lc[2]);
                for (int j = 0; j < s.m; ++j) out[(size_t)j * s.N + lex] = tmp[(size_t)j * s.N + c];
            }
            return MRCM_OK;
        }
        default: return fail(h, MRCM_ERR_INVALID_ARG, "unknown export");
    }
    if (bytes < need) return fail(h, MRCM_ERR_INVALID_ARG, "export buffer too small");
    e = cudaMemcpy(dst, src, need, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "mrcm_export");
    return MRCM_OK;
}

mrcm_status mrcm_query_tuning(const mrcm_handle* h, int* solve_variant, int* sweep_variant, int* factor_small,
                              int* factor_mid) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    if (solve_variant) *solve_variant = h->d.solve_variant;
    if (sweep_variant) *sweep_variant = h->d.sweep_variant;
    if (factor_small) *factor_small = h->d.factor_variant;
    if (factor_mid) *factor_mid = h->d.factor_mid_variant;
    return MRCM_OK;
}

mrcm_status mrcm_read_tuning_times(const mrcm_handle* h, float* solve_ms, float* sweep_ms, int* solve_ctas,
                                   int* sweep_ctas, int cap, int* n, int* sweeps_separate, float* sweeps_separate_ms) {
    if (!h || cap < 0) return MRCM_ERR_INVALID_ARG;
    if (n) *n = h->tune_n;
    if (sweeps_separate) *sweeps_separate = h->d.sweeps_separate;
    if (sweeps_separate_ms) *sweeps_separate_ms = h->d.sweeps_separate_ms;
    for (int v = 0; v < h->tune_n && v < cap; ++v) {
        if (solve_ms) solve_ms[v] = h->tune_ms[2 * v];
        if (sweep_ms) sweep_ms[v] = h->tune_ms[2 * v + 1];
        if (solve_ctas) solve_ctas[v] = h->d.solve_occ[v];
        if (sweep_ctas) sweep_ctas[v] = h->d.sweep_occ[v];
    }
    return MRCM_OK;
}

mrcm_status mrcm_autotune(mrcm_handle* h, const double* f, void* ws, void* stream, int* solve_variant,
                          int* sweep_variant) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    if (!f) return fail(h, MRCM_ERR_INVALID_ARG, "f is NULL");
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    if (h->stage < 1) return fail(h, MRCM_ERR_STATE, "mrcm_factor_local must run first");
    if (h->t.cfg.precision == MRCM_LEARNED_PCG) return fail(h, MRCM_ERR_INVALID_ARG, "the learned form has no direct solve to tune");
    int v0 = 0, v1 = 0, v2 = h->d.factor_variant, v3 = h->d.factor_mid_variant;
    float ms[2 * mrcm::kMaxSolveVariants];
    for (float& x : ms) x = -1.0f;
    int rc = mrcm::autotune_local(h->t, h->d, h->lay, (char*)ws, f, stream, 3, &v0, &v1, &v2, &v3, ms);
    if ((st = after_launch(h, rc, "mrcm_autotune")) != MRCM_OK) return st;
    for (int i = 0; i < 2 * mrcm::kMaxSolveVariants; ++i) h->tune_ms[i] = ms[i];
    h->tune_n = mrcm::num_solve_variants();
    h->d.solve_variant = v0;
    h->d.sweep_variant = v1;
    h->d.factor_variant = v2;
    h->d.factor_mid_variant = v3;
    drop_graph(h);                       // a captured graph holds the old variants
    store_tune_cache(h);
    h->stage = 1;                        // the tuning runs overwrote the MBF array
    if (solve_variant) *solve_variant = v0;
    if (sweep_variant) *sweep_variant = v1;
    return MRCM_OK;
}

static mrcm_status run_all(mrcm_handle* h, const double* K, const double* f, double* X, double* p, double* u,
                           double* mres, void* ws, size_t ws_bytes, void* stream) {
    mrcm_status st;
    if ((st = mrcm_factor_local(h, K, ws, ws_bytes, stream)) != MRCM_OK) return st;
    if ((st = mrcm_solve_mbf(h, f, ws, stream)) != MRCM_OK) return st;
    if ((st = mrcm_assemble_interface(h, ws, stream)) != MRCM_OK) return st;
    if ((st = mrcm_solve_interface(h, X, ws, stream)) != MRCM_OK) return st;
    return mrcm_reconstruct(h, X, p, u, mres, ws, stream);
}

mrcm_status mrcm_solve(mrcm_handle* h, const double* K, const double* f, double* X, double* p, double* u,
                       double* mres, void* ws, size_t ws_bytes, void* stream, int flags) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    if (!(flags & MRCM_SOLVE_GRAPH)) return run_all(h, K, f, X, p, u, mres, ws, ws_bytes, stream);
    if (!stream) return fail(h, MRCM_ERR_INVALID_ARG, "graph mode needs a non-default stream");
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    if (ws_bytes < h->lay.total) return fail(h, MRCM_ERR_OOM, "workspace smaller than mrcm_query_workspace");
    if ((st = ensure_device(h, stream)) != MRCM_OK) return st;
    const void* key[9] = {K, f, X, p, u, mres, ws, stream, (const void*)(size_t)ws_bytes};
    bool same = h->graph_exec != nullptr;
    for (int i = 0; i < 9 && same; ++i) same = key[i] == h->graph_key[i];
    cudaError_t e;
    if (!same) {
        drop_graph(h);
        const bool prof = h->prof.on;
        h->prof.on = false;
        const long long n0 = h->prof.launches;
        e = cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { h->prof.on = prof; return cuda_fail(h, e, "cudaStreamBeginCapture"); }
        mrcm_status rs = run_all(h, K, f, X, p, u, mres, ws, ws_bytes, stream);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture((cudaStream_t)stream, &g);
        h->prof.on = prof;
        h->graph_launches = h->prof.launches - n0;
        h->prof.launches = n0;
        if (rs != MRCM_OK) { if (g) cudaGraphDestroy(g); return rs; }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        h->graph = g;
        e = cudaGraphInstantiate(&h->graph_exec, g, 0);
        if (e != cudaSuccess) { drop_graph(h); return cuda_fail(h, e, "cudaGraphInstantiate"); }
        for (int i = 0; i < 9; ++i) h->graph_key[i] = key[i];
    }
    e = cudaGraphLaunch(h->graph_exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
    h->prof.launches += h->graph_launches;
    h->stage = 4;
    return MRCM_OK;
}

// Host-buffer solve: inputs copied in (K in two halves, one on a side stream
// with f), the solve, outputs copied out (u in two halves, p on the side
// stream); graph mode captures copies and solve into one CUDA graph.
static mrcm_status host_body(mrcm_handle* h, const double* K, const double* f, double* X, double* p, double* u,
                             double* mres, void* ws, size_t ws_bytes, cudaStream_t st) {
    const size_t nc = (size_t)h->t.n_cells, nx = (size_t)std::max(2 * h->t.NV, 1);
    double* dK = h->io;
    double* df = dK + 3 * nc;
    double* dX = df + nc;
    double* dp = dX + nx;
    double* du = dp + nc;
    double* dm = du + 6 * nc;
    cudaStream_t sd = h->io_side;
    const size_t kh = (3 * nc) / 2, uh = (6 * nc) / 2;
    cudaEventRecord(h->io_ev[0], st);
    cudaStreamWaitEvent(sd, h->io_ev[0], 0);
    cudaMemcpyAsync(dK, K, kh * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dK + kh, K + kh, (3 * nc - kh) * sizeof(double), cudaMemcpyHostToDevice, sd);
    cudaMemcpyAsync(df, f, nc * sizeof(double), cudaMemcpyHostToDevice, sd);
    cudaEventRecord(h->io_ev[1], sd);
    cudaStreamWaitEvent(st, h->io_ev[1], 0);
    mrcm_status rs = run_all(h, dK, df, dX, dp, du, dm, ws, ws_bytes, st);
    if (rs != MRCM_OK) return rs;
    cudaEventRecord(h->io_ev[0], st);
    cudaStreamWaitEvent(sd, h->io_ev[0], 0);
    cudaMemcpyAsync(u, du, uh * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(u + uh, du + uh, (6 * nc - uh) * sizeof(double), cudaMemcpyDeviceToHost, sd);
    cudaMemcpyAsync(p, dp, nc * sizeof(double), cudaMemcpyDeviceToHost, sd);
    cudaMemcpyAsync(X, dX, 2 * (size_t)h->t.NV * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (mres) cudaMemcpyAsync(mres, dm, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaEventRecord(h->io_ev[1], sd);
    cudaStreamWaitEvent(st, h->io_ev[1], 0);
    return MRCM_OK;
}

mrcm_status mrcm_solve_host(mrcm_handle* h, const double* K, const double* f, double* X, double* p, double* u,
                            double* mres, void* ws, size_t ws_bytes, void* stream, int flags) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    mrcm_status st = check_ws(h, ws);
    if (st != MRCM_OK) return st;
    if (!K || !f || !X || !p || !u) return fail(h, MRCM_ERR_INVALID_ARG, "K, f, X, p and u must be non-NULL");
    if (!stream) return fail(h, MRCM_ERR_INVALID_ARG, "the host-buffer solve needs a non-default stream");
    if (ws_bytes < h->lay.total) return fail(h, MRCM_ERR_OOM, "workspace smaller than mrcm_query_workspace");
    if ((st = ensure_device(h, stream)) != MRCM_OK) return st;
    cudaError_t e;
    if (!h->io) {
        const size_t nc = (size_t)h->t.n_cells, nx = (size_t)std::max(2 * h->t.NV, 1);
        h->io_bytes = (11 * nc + nx + 1) * sizeof(double);
        if ((e = cudaMalloc(&h->io, h->io_bytes)) != cudaSuccess) { h->io = nullptr; return cuda_fail(h, e, "cudaMalloc (staging)"); }
    }
    // side stream and events: created once; a call after a failed creation retries it
    if (!h->io_side && (e = cudaStreamCreateWithFlags(&h->io_side, cudaStreamNonBlocking)) != cudaSuccess) {
        h->io_side = nullptr;
        return cuda_fail(h, e, "cudaStreamCreate");
    }
    for (auto& ev : h->io_ev)
        if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            ev = nullptr;
            return cuda_fail(h, e, "cudaEventCreate");
        }
    cudaStream_t s = (cudaStream_t)stream;
    if (!(flags & MRCM_SOLVE_GRAPH)) {
        st = host_body(h, K, f, X, p, u, mres, ws, ws_bytes, s);
        if (st != MRCM_OK) return st;
        e = cudaGetLastError();
        return e == cudaSuccess ? MRCM_OK : cuda_fail(h, e, "mrcm_solve_host");
    }
    const void* key[10] = {K, f, X, p, u, mres, ws, stream, (const void*)(size_t)ws_bytes, (const void*)1};
    bool same = h->hgraph_exec != nullptr;
    for (int i = 0; i < 10 && same; ++i) same = key[i] == h->hgraph_key[i];
    if (!same) {
        if (h->hgraph_exec) cudaGraphExecDestroy(h->hgraph_exec);
        if (h->hgraph) cudaGraphDestroy(h->hgraph);
        h->hgraph_exec = nullptr;
        h->hgraph = nullptr;
        const bool prof = h->prof.on;
        h->prof.on = false;
        const long long n0 = h->prof.launches;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { h->prof.on = prof; return cuda_fail(h, e, "cudaStreamBeginCapture"); }
        mrcm_status rs = host_body(h, K, f, X, p, u, mres, ws, ws_bytes, s);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(s, &g);
        h->prof.on = prof;
        h->hgraph_launches = h->prof.launches - n0;
        h->prof.launches = n0;
        if (rs != MRCM_OK) { if (g) cudaGraphDestroy(g); return rs; }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture (host buffers must be pinned)");
        h->hgraph = g;
        e = cudaGraphInstantiate(&h->hgraph_exec, g, 0);
        if (e != cudaSuccess) { cudaGraphDestroy(g); h->hgraph = nullptr; h->hgraph_exec = nullptr; return cuda_fail(h, e, "cudaGraphInstantiate"); }
        for (int i = 0; i < 10; ++i) h->hgraph_key[i] = key[i];
    }
    e = cudaGraphLaunch(h->hgraph_exec, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
    h->prof.launches += h->hgraph_launches;
    h->stage = 4;
    return MRCM_OK;
}

mrcm_status mrcm_profile(mrcm_handle* h, int enable) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    h->prof.reset();
    h->prof.on = enable != 0;
    return MRCM_OK;
}

mrcm_status mrcm_profile_report(mrcm_handle* h, char* buf, size_t len, long long* launches) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    mrcm::Prof& P = h->prof;
    if (launches) *launches = P.launches;
    std::vector<double> ms(P.names.size(), 0.0);
    std::vector<long long> cnt(P.names.size(), 0);
    if (P.used) {
        cudaError_t e = cudaEventSynchronize(P.pool[P.used - 1]);
        if (e != cudaSuccess) return cuda_fail(h, e, "mrcm_profile_report");
    }
    for (size_t i = 0; i < P.kid.size(); ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, P.pool[2 * i], P.pool[2 * i + 1]) == cudaSuccess) {
            ms[P.kid[i]] += t;
            cnt[P.kid[i]] += 1;
        }
    }
    std::string out;
    for (size_t k = 0; k < P.names.size(); ++k) {
        if (!cnt[k]) continue;
        char line[256];
        snprintf(line, sizeof(line), "%s %lld %.6f\n", P.names[k].c_str(), cnt[k], ms[k]);
        out += line;
    }
    if (buf && len) {
        size_t n = std::min(len - 1, out.size());
        std::memcpy(buf, out.data(), n);
        buf[n] = 0;
        if (out.size() >= len) return fail(h, MRCM_ERR_INVALID_ARG, "profile buffer too small");
    }
    P.reset();
    return MRCM_OK;
}

void mrcm_destroy(mrcm_handle* h) {
    if (!h) return;
    h->prof.release();
    drop_graph(h);
    if (h->hgraph_exec) cudaGraphExecDestroy(h->hgraph_exec);
    if (h->hgraph) cudaGraphDestroy(h->hgraph);
    if (h->io) cudaFree(h->io);
    if (h->io_side) cudaStreamDestroy(h->io_side);
    for (auto ev : h->io_ev) if (ev) cudaEventDestroy(ev);
    if (h->samp_off) cudaFree(h->samp_off);
    if (h->samp_list) cudaFree(h->samp_list);
    if (h->col_list) cudaFree(h->col_list);
    free_device(h->d);
    delete h;
}

const char* mrcm_last_error(const mrcm_handle* h) {
    if (!h) return g_setup_err.c_str();
    return h->err.c_str();
}

}  // extern "C"
