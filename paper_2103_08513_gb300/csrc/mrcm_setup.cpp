// Host-side setup of libmrcm: decomposition, interface space, Robin faces,
// per-subdomain right-hand-side layout, interface CSR pattern and the
// nested-dissection elimination tree of the interface system.
//
// Decomposition and interface space: Sec. "Domain decomposition and Darcy
// solvers" and Sec. "A domain decomposition Multiscale Mixed method" of the
// paper (patch basis functions of Fig. decomposition_h_H, counted by
// Eq. dof_PH).  The elimination tree is this library's own design (the paper
// uses MUMPS with the PORD ordering for the interface system).
#include <algorithm>
#include <cstring>
#include <map>
#include <unordered_map>

#include "mrcm_internal.h"

namespace mrcm {

namespace {

struct Box { int lo[3], hi[3]; };

struct TreeBuilder {
    Tables& t;
    std::vector<std::vector<int>> Bsets;   // per internal node: boundary bases (sorted)
    explicit TreeBuilder(Tables& tt) : t(tt) {}

    int sub_index(int ix, int iy, int iz) const { return ix + t.N[0] * (iy + t.N[1] * iz); }

    // Boundary bases of a child: the leaf's I^l, or the internal node's B.
    const std::vector<int>& child_B(int c, std::vector<int>& tmp) {
        if (c < 0) {
            const SubInfo& s = t.subs[-(c + 1)];
            tmp.assign(t.Ilist.begin() + s.I_off, t.Ilist.begin() + s.I_off + s.nI);
            return tmp;
        }
        return Bsets[c];
    }

    int build(const Box& bx) {
        int ext[3], tot = 1;
        for (int a = 0; a < 3; ++a) { ext[a] = bx.hi[a] - bx.lo[a]; tot *= ext[a]; }
        if (tot == 1) return -(1 + sub_index(bx.lo[0], bx.lo[1], bx.lo[2]));
        int ax = 0;
        for (int a = 1; a < 3; ++a) if (ext[a] > ext[ax]) ax = a;
        Box L = bx, R = bx;
        int mid = bx.lo[ax] + ext[ax] / 2;
        L.hi[ax] = mid;
        R.lo[ax] = mid;
        int c0 = build(L);
        int c1 = build(R);
        std::vector<int> t0, t1;
        const std::vector<int>& B0 = child_B(c0, t0);
        const std::vector<int>& B1 = child_B(c1, t1);
        std::vector<int> E, B;
        std::set_intersection(B0.begin(), B0.end(), B1.begin(), B1.end(), std::back_inserter(E));
        std::set_symmetric_difference(B0.begin(), B0.end(), B1.begin(), B1.end(), std::back_inserter(B));
        FrontInfo fi;
        std::memset(&fi, 0, sizeof(fi));
        fi.ne = 2 * (int)E.size();
        fi.nb = 2 * (int)B.size();
        fi.n = fi.ne + fi.nb;
        fi.nchild = 2;
        fi.child[0] = c0;
        fi.child[1] = c1;
        fi.pin_row = -1;
        fi.parent = -1;
        auto h = [&](int c) { return c < 0 ? 0 : t.fronts[c].height; };
        fi.height = 1 + std::max(h(c0), h(c1));
        fi.e_dof_off = (int)t.front_dofs.size();
        for (int k : E) t.front_dofs.push_back(k);
        for (int k : E) t.front_dofs.push_back(t.NV + k);
        for (int k : B) t.front_dofs.push_back(k);
        for (int k : B) t.front_dofs.push_back(t.NV + k);
        int id = (int)t.fronts.size();
        t.fronts.push_back(fi);
        Bsets.push_back(B);
        if (c0 >= 0) t.fronts[c0].parent = id;
        if (c1 >= 0) t.fronts[c1].parent = id;
        return id;
    }
};

}  // namespace

mrcm_status build_tables(const mrcm_config* cfg, Tables& t, std::string& err) {
    if (!cfg) { err = "config is NULL"; return MRCM_ERR_INVALID_ARG; }
    if (cfg->interface_refine < -1) { err = "interface_refine must be >= -1"; return MRCM_ERR_INVALID_ARG; }
    if (cfg->fallback_cap < -1) { err = "fallback_cap must be >= -1"; return MRCM_ERR_INVALID_ARG; }
    t.cfg = *cfg;
    if (cfg->tune_cache) t.tune_cache = cfg->tune_cache;
    t.cfg.tune_cache = nullptr;
    const int n[3] = {cfg->nx, cfg->ny, cfg->nz};
    const double hh[3] = {cfg->hx, cfg->hy, cfg->hz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1) { err = "grid extents must be >= 1"; return MRCM_ERR_INVALID_ARG; }
        if (!(hh[a] > 0)) { err = "cell sizes must be > 0"; return MRCM_ERR_INVALID_ARG; }
        if (cfg->n_cuts[a] < 1 || !cfg->cuts[a]) { err = "each axis needs an edge list"; return MRCM_ERR_INVALID_ARG; }
        t.cuts[a].assign(cfg->cuts[a], cfg->cuts[a] + cfg->n_cuts[a]);
        long long s = 0;
        for (int e : t.cuts[a]) {
            if (e < 1) { err = "subdomain edges must be >= 1"; return MRCM_ERR_INVALID_ARG; }
            s += e;
        }
        if (s != n[a]) { err = "edge list of axis " + std::to_string(a) + " does not sum to the grid extent"; return MRCM_ERR_INVALID_ARG; }
        t.N[a] = cfg->n_cuts[a];
        t.starts[a].assign(1, 0);
        for (int e : t.cuts[a]) t.starts[a].push_back(t.starts[a].back() + e);
        for (int s2 = 0; s2 < 2; ++s2) {
            if (cfg->patch[a][s2] < 0) { err = "patch sizes must be >= 0"; return MRCM_ERR_INVALID_ARG; }
            if (cfg->bc_type[a][s2] != MRCM_BC_NOFLOW && cfg->bc_type[a][s2] != MRCM_BC_DIRICHLET) {
                err = "unknown wall condition"; return MRCM_ERR_INVALID_ARG;
            }
            if (cfg->bc_type[a][s2] == MRCM_BC_DIRICHLET) t.has_dirichlet = true;
        }
    }
    if (cfg->beta_mode != MRCM_BETA_CONST && cfg->beta_mode != MRCM_BETA_ALPHA_H_OVER_K) {
        err = "unknown beta mode"; return MRCM_ERR_INVALID_ARG;
    }
    if (cfg->beta_mode == MRCM_BETA_CONST && !(cfg->beta_const > 0)) { err = "beta must be > 0"; return MRCM_ERR_INVALID_ARG; }
    if (cfg->beta_mode == MRCM_BETA_ALPHA_H_OVER_K && !(cfg->alpha > 0)) { err = "alpha must be > 0"; return MRCM_ERR_INVALID_ARG; }
    if (cfg->precision < MRCM_FP64 || cfg->precision > MRCM_LEARNED_PCG) { err = "unknown precision"; return MRCM_ERR_INVALID_ARG; }
    if (cfg->ir_max_sweeps < 0 || cfg->ir_max_sweeps > 64) { err = "ir_max_sweeps must be in [0, 64]"; return MRCM_ERR_INVALID_ARG; }
    const int nsub = t.N[0] * t.N[1] * t.N[2];
    if (nsub == 1 && !t.has_dirichlet) {
        err = "one subdomain with no-flow walls leaves the pressure undetermined";
        return MRCM_ERR_INVALID_ARG;
    }
    t.n_cells = (long long)n[0] * n[1] * n[2];

    // ---- subdomains --------------------------------------------------------
    t.subs.resize(nsub);
    for (int iz = 0; iz < t.N[2]; ++iz)
        for (int iy = 0; iy < t.N[1]; ++iy)
            for (int ix = 0; ix < t.N[0]; ++ix) {
                int l = ix + t.N[0] * (iy + t.N[1] * iz);
                SubInfo& s = t.subs[l];
                std::memset(&s, 0, sizeof(s));
                const int id[3] = {ix, iy, iz};
                for (int a = 0; a < 3; ++a) { s.o[a] = t.starts[a][id[a]]; s.sz[a] = t.cuts[a][id[a]]; }
                // slab axis: the longest; ties go to the higher axis so that x stays in-slab
                int sa = 2;
                for (int a = 1; a >= 0; --a) if (s.sz[a] > s.sz[sa]) sa = a;
                s.sa = sa;
                s.ua = sa == 0 ? 1 : 0;
                s.va = sa == 2 ? 1 : 2;
                s.su = s.sz[s.ua];
                s.sv = s.sz[s.va];
                s.b = s.su * s.sv;
                s.ns = s.sz[sa];
                s.N = s.b * s.ns;
                s.big_slot = -1;
                const int bmax = kMaxBlock;
                if (s.b > bmax) {
                    err = "subdomain slab block " + std::to_string(s.b) + " exceeds " + std::to_string(bmax);
                    return MRCM_ERR_NOT_IMPLEMENTED;
                }
            }

    // ---- basis functions (canonical order) ---------------------------------
    std::vector<std::vector<int>> I(nsub);
    struct BFace { int clo_loc_lo; int clo_loc_hi; };
    std::vector<std::vector<std::pair<int,int>>> bfaces;   // per basis: (local cell in lo, local cell in hi)
    auto local_index = [&](const SubInfo& s, const int g[3]) {
        int c[3] = {g[0] - s.o[0], g[1] - s.o[1], g[2] - s.o[2]};
        return c[s.sa] * s.b + c[s.ua] + s.su * c[s.va];
    };
    for (int a = 0; a < 3; ++a) {
        int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
        for (int l = 0; l < nsub; ++l) {
            int id[3] = {l % t.N[0], (l / t.N[0]) % t.N[1], l / (t.N[0] * t.N[1])};
            if (id[a] == t.N[a] - 1) continue;
            int id2[3] = {id[0], id[1], id[2]};
            id2[a] += 1;
            int l2 = id2[0] + t.N[0] * (id2[1] + t.N[1] * id2[2]);
            int lo1 = t.starts[t1][id[t1]], E1 = t.cuts[t1][id[t1]];
            int lo2 = t.starts[t2][id[t2]], E2 = t.cuts[t2][id[t2]];
            int p1 = cfg->patch[a][0], p2 = cfg->patch[a][1];
            p1 = p1 == 0 ? E1 : std::min(p1, E1);
            p2 = p2 == 0 ? E2 : std::min(p2, E2);
            int n1 = (E1 + p1 - 1) / p1, n2 = (E2 + p2 - 1) / p2;
            int xa = t.starts[a][id[a] + 1];
            for (int q2 = 0; q2 < n2; ++q2)
                for (int q1 = 0; q1 < n1; ++q1) {
                    int k = t.NV++;
                    t.b_axis.push_back(a);
                    t.b_lo.push_back(l);
                    t.b_hi.push_back(l2);
                    std::vector<std::pair<int,int>> fl;
                    for (int c2 = lo2 + q2 * p2; c2 < std::min(lo2 + (q2 + 1) * p2, lo2 + E2); ++c2)
                        for (int c1 = lo1 + q1 * p1; c1 < std::min(lo1 + (q1 + 1) * p1, lo1 + E1); ++c1) {
                            int g[3];
                            g[a] = xa - 1; g[t1] = c1; g[t2] = c2;
                            int cl = local_index(t.subs[l], g);
                            g[a] = xa;
                            int ch = local_index(t.subs[l2], g);
                            fl.push_back({cl, ch});
                        }
                    t.b_nfaces.push_back((int)fl.size());
                    bfaces.push_back(std::move(fl));
                    I[l].push_back(k);
                    I[l2].push_back(k);
                }
        }
    }

    // ---- per-subdomain lists and offsets -------------------------------------
    long long cell_off = 0, x_off = 0, el_off = 0;
    int elb_off = 0;
    for (int l = 0; l < nsub; ++l) {
        SubInfo& s = t.subs[l];
        std::sort(I[l].begin(), I[l].end());
        s.nI = (int)I[l].size();
        s.m = 2 * s.nI + 1;
        s.el_dim = 2 * s.nI;
        s.I_off = (int)t.Ilist.size();
        t.Ilist.insert(t.Ilist.end(), I[l].begin(), I[l].end());
        s.face_off = (int)t.faces.size();
        for (int c = 0; c < s.nI; ++c) {
            int k = I[l][c];
            bool lo = t.b_lo[k] == l;
            for (auto& pr : bfaces[k]) {
                FaceInfo fi;
                fi.cell = lo ? pr.first : pr.second;
                fi.col = c;
                fi.axis = (int8_t)t.b_axis[k];
                fi.s = lo ? 1 : -1;
                fi.pad = 0;
                t.faces.push_back(fi);
            }
        }
        s.nface = (int)t.faces.size() - s.face_off;
        s.cell_off = cell_off;  cell_off += s.N;
        s.x_off = x_off;        s.y_off = x_off;        x_off += (long long)s.m * s.N;
        s.el_off = el_off;      el_off += (long long)s.el_dim * s.el_dim;
        s.elb_off = elb_off;    elb_off += s.el_dim;
        s.rhs_off = (int)t.total_rhs;
        t.max_m = std::max(t.max_m, s.m);
        t.max_b = std::max(t.max_b, s.b);
        t.max_el = std::max(t.max_el, s.el_dim);
        t.max_N = std::max(t.max_N, s.N);
        t.total_rhs += s.m;
        t.local_factor_flops += (double)s.N * s.b * s.b;    // banded-Cholesky count of the block factor
        t.local_solve_flops += 4.0 * s.N * (double)s.b * s.m;
    }
    // solve order (costliest first), memory-bounded waves over it, and per wave the
    // factor classes (register-resident FP32 factor for small blocks), costliest first
    {
        std::vector<std::pair<double, int>> sl;
        for (int l = 0; l < nsub; ++l) {
            const SubInfo& s = t.subs[l];
            sl.push_back({-(double)s.N * s.b * s.m, l});
        }
        std::sort(sl.begin(), sl.end());
        for (auto& pr : sl) t.solve_list.push_back(pr.second);
        const size_t welem = cfg->precision == MRCM_FP64 ? sizeof(double) : sizeof(float);
        t.wave_off.assign(1, 0);
        long long wcur = 0, wmax = 0;
        for (int q = 0; q < nsub; ++q) {
            SubInfo& s = t.subs[t.solve_list[q]];
            const long long need = (long long)s.ns * (t.cfg.precision == MRCM_FP64 ? wstride<double>(s.b) : wstride<float>(s.b));
            if (cfg->wave_bytes > 0 && q > t.wave_off.back() && (size_t)(wcur + need) * welem > cfg->wave_bytes) {
                t.wave_off.push_back(q);
                wcur = 0;
            }
            s.w_off = wcur;
            wcur += need;
            wmax = std::max(wmax, wcur);
        }
        t.wave_off.push_back(nsub);
        t.n_waves = (int)t.wave_off.size() - 1;
        t.total_w = wmax;
        // FP64 form: blocks above kMaxBlock64 keep their packed triangle in a global slot
        if (cfg->precision == MRCM_FP64) {
            for (int w = 0; w < t.n_waves; ++w) {
                int k = 0;
                for (int q = t.wave_off[w]; q < t.wave_off[w + 1]; ++q) {
                    SubInfo& s = t.subs[t.solve_list[q]];
                    if (s.b > kMaxBlock64) s.big_slot = k++;
                }
                t.big_slots = std::max(t.big_slots, k);
            }
        }
        t.class_list.clear();
        for (int w = 0; w < t.n_waves; ++w) {
            std::vector<std::tuple<int, double, int>> cls[3];
            for (int q = t.wave_off[w]; q < t.wave_off[w + 1]; ++q) {
                const int l = t.solve_list[q];
                const SubInfo& s = t.subs[l];
                const double cost = (double)s.ns * s.b * s.b * s.b;
                const int k = cfg->precision == MRCM_FP64 ? 2 : s.b <= kRegBlock ? 0 : s.b <= kTileBlock ? 1 : 2;
                // mixed large class: ordered by b first (its factor launches
                // one CTA size per run of b), then by cost
                cls[k].push_back({k == 2 && cfg->precision != MRCM_FP64 ? -s.b : 0, -cost, l});
            }
            for (int k = 0; k < 3; ++k) {
                std::sort(cls[k].begin(), cls[k].end());
                t.wave_class_off.push_back((int)t.class_list.size());
                for (auto& e : cls[k]) t.class_list.push_back(std::get<2>(e));
            }
            t.wave_class_off.push_back((int)t.class_list.size());
        }
        for (int k = 0; k < 4; ++k) t.class_off[k] = t.wave_class_off[k];
        // FP64 post-processing waves of the mixed modes (the W region holds total_w floats)
        if (cfg->precision != MRCM_FP64) {
            t.pp_subs = t.subs;
            t.pp_wave_off.assign(1, 0);
            const long long cap_d = t.total_w * (long long)sizeof(float) / (long long)sizeof(double);
            long long cur = 0;
            for (int q = 0; q < nsub; ++q) {
                SubInfo& s = t.pp_subs[t.solve_list[q]];
                const long long need = (long long)s.ns * wstride<double>(s.b);
                if (s.b > kMaxBlock64 || need > cap_d) t.pp_ok = false;
                if (q > t.pp_wave_off.back() && cur + need > cap_d) {
                    t.pp_wave_off.push_back(q);
                    cur = 0;
                }
                s.w_off = cur;
                s.y_off = s.cell_off;      // one column of forward values per cell
                cur += need;
            }
            t.pp_wave_off.push_back(nsub);
        }
    }
    t.total_x = x_off;
    t.total_el = el_off;
    t.total_elb = elb_off;

    // ---- interface CSR pattern with two-sided sources --------------------------
    const int nd = 2 * t.NV;
    t.rowptr.assign(1, 0);
    t.rhs_src_lo.assign(nd, -1);
    t.rhs_src_hi.assign(nd, -1);
    auto elem_row = [&](int l, int dof) {   // position of global dof in element l, or -1
        const SubInfo& s = t.subs[l];
        int k = dof < t.NV ? dof : dof - t.NV;
        auto it = std::lower_bound(I[l].begin(), I[l].end(), k);
        if (it == I[l].end() || *it != k) return -1;
        int c = (int)(it - I[l].begin());
        return dof < t.NV ? c : s.nI + c;
    };
    auto elem_dof = [&](int l, int e) {
        const SubInfo& s = t.subs[l];
        return e < s.nI ? I[l][e] : t.NV + I[l][e - s.nI];
    };
    for (int r = 0; r < nd; ++r) {
        int k = r < t.NV ? r : r - t.NV;
        std::map<int, std::pair<long long, long long>> cols;
        for (int side = 0; side < 2; ++side) {
            int l = side == 0 ? t.b_lo[k] : t.b_hi[k];
            const SubInfo& s = t.subs[l];
            int er = elem_row(l, r);
            if (side == 0) t.rhs_src_lo[r] = s.elb_off + er; else t.rhs_src_hi[r] = s.elb_off + er;
            for (int e = 0; e < s.el_dim; ++e) {
                int gc = elem_dof(l, e);
                auto& pr = cols.emplace(gc, std::make_pair(-1LL, -1LL)).first->second;
                long long off = s.el_off + (long long)er * s.el_dim + e;
                if (side == 0) pr.first = off; else pr.second = off;
            }
        }
        for (auto& kv : cols) {
            t.colidx.push_back(kv.first);
            t.src_lo.push_back(kv.second.first);
            t.src_hi.push_back(kv.second.second);
        }
        t.rowptr.push_back((int)t.colidx.size());
    }

    // ---- nested-dissection elimination tree ----------------------------------
    if (nsub > 1) {
        TreeBuilder tb(t);
        Box all;
        for (int a = 0; a < 3; ++a) { all.lo[a] = 0; all.hi[a] = t.N[a]; }
        t.root = tb.build(all);
        int maxh = 0;
        for (auto& f : t.fronts) maxh = std::max(maxh, f.height);
        t.levels.assign(maxh + 1, {});
        long long foff = 0;
        int roff = 0;
        for (int id = 0; id < (int)t.fronts.size(); ++id) {
            FrontInfo& f = t.fronts[id];
            t.levels[f.height].push_back(id);
            f.f_off = foff;  foff += (long long)f.n * f.n;
            f.r_off = roff;  roff += f.n;
            f.p_off = t.total_panels;  t.total_panels += (f.ne + 31) / 32;
            t.max_front = std::max(t.max_front, f.n);
            for (int k0 = 0; k0 < f.ne; k0 += 32) {
                const double nbk = std::min(32, f.ne - k0);
                const double mrem = f.n - k0 - nbk;
                t.ldl_update_flops += nbk * mrem * (mrem + 1.0);
            }
            for (int kk = 0; kk < f.ne; ++kk) {
                double rem = f.n - kk - 1;
                t.front_flops += rem + 2.0 * rem * rem;
                t.ldl_flops += rem + rem * (rem + 1.0);
            }
            std::unordered_map<int, int> pos;
            for (int q = 0; q < f.n; ++q) pos[t.front_dofs[f.e_dof_off + q]] = q;
            f.inv_off = (int)t.front_inv.size();
            t.front_inv.resize(t.front_inv.size() + 2 * (size_t)f.n, -1);
            for (int ci = 0; ci < 2; ++ci) {
                int c = f.child[ci];
                f.map_off[ci] = (int)t.front_maps.size();
                if (c < 0) {
                    int l = -(c + 1);
                    const SubInfo& s = t.subs[l];
                    for (int e = 0; e < s.el_dim; ++e) t.front_maps.push_back(pos.at(elem_dof(l, e)));
                    f.map_len[ci] = s.el_dim;
                } else {
                    const FrontInfo& cf = t.fronts[c];
                    for (int q = cf.ne; q < cf.n; ++q) t.front_maps.push_back(pos.at(t.front_dofs[cf.e_dof_off + q]));
                    f.map_len[ci] = cf.nb;
                }
                for (int q = 0; q < f.map_len[ci]; ++q)
                    t.front_inv[f.inv_off + (size_t)ci * f.n + t.front_maps[f.map_off[ci] + q]] = q;
            }
            if (!t.has_dirichlet && t.NV > 0) {
                auto it = pos.find(0);
                if (it != pos.end() && it->second < f.ne) { f.pin_row = it->second; t.pin_front = id; }
            }
        }
        for (const auto& lv : t.levels) {
            long long rows = 0;
            for (int id : lv) {
                FrontInfo& f = t.fronts[id];
                f.s_off = -1;
                if (f.n >= kOzMinN) { f.s_off = (int)rows; rows += f.n; }
            }
            t.oz_rows = std::max(t.oz_rows, rows);
        }
        for (const FrontInfo& f : t.fronts) {         // BF16 work of the steps the update emulates
            if (f.s_off < 0) continue;
            for (int k0 = 0; k0 < f.ne; k0 += 32) {
                const int nbk = std::min(32, f.ne - k0), m = f.n - k0 - nbk;
                if (m < kOzMinM || nbk < kOzMinK) continue;
                const double nt = (m + 31) / 32;
                t.ldl_update_tensor_flops += nt * (nt + 1.0) / 2.0 * kOzTileFlops;
            }
        }
        t.total_front = foff;
        t.total_frhs = roff;
        if (t.root < 0 || t.fronts[t.root].nb != 0) { err = "internal: elimination tree root keeps boundary dofs"; return MRCM_ERR_INVALID_ARG; }
    }
    return MRCM_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Algorithmic cost of a sparse direct LDL^T of one box's local matrix (the
// paper's local solver, Sec. "MBFs: LocalSolver()"): exact minimum degree on
// the 7-point graph (ties: lowest box-lexicographic index), the neighbour
// count c_j at elimination = below-diagonal entries of column j of L;
// factor flops sum c_j (c_j + 3), nnz(L) = sum c_j.  Bitset rows (n <= 4096).
void min_degree_cost(int sx, int sy, int sz, double* flops, long long* nnz) {
    const int n = sx * sy * sz, W = (n + 63) / 64;
    std::vector<uint64_t> G((size_t)n * W, 0ull);
    auto setb = [&](int a, int b) { G[(size_t)a * W + b / 64] |= 1ull << (b % 64); };
    for (int k = 0; k < sz; ++k)
        for (int j = 0; j < sy; ++j)
            for (int i = 0; i < sx; ++i) {
                const int c = i + sx * (j + sy * k);
                if (i + 1 < sx) { setb(c, c + 1); setb(c + 1, c); }
                if (j + 1 < sy) { setb(c, c + sx); setb(c + sx, c); }
                if (k + 1 < sz) { setb(c, c + sx * sy); setb(c + sx * sy, c); }
            }
    auto popc = [&](int a) {
        int d = 0;
        for (int w = 0; w < W; ++w) d += __builtin_popcountll(G[(size_t)a * W + w]);
        return d;
    };
    std::vector<int> deg(n);
    std::vector<char> alive(n, 1);
    for (int a = 0; a < n; ++a) deg[a] = popc(a);
    double fl = 0.0;
    long long nz = 0;
    std::vector<int> nb;
    for (int step = 0; step < n; ++step) {
        int v = -1;
        for (int a = 0; a < n; ++a)
            if (alive[a] && (v < 0 || deg[a] < deg[v])) v = a;
        const long long c = deg[v];
        fl += (double)c * (double)(c + 3);
        nz += c;
        nb.clear();
        for (int w = 0; w < W; ++w) {
            uint64_t x = G[(size_t)v * W + w];
            while (x) { nb.push_back(w * 64 + __builtin_ctzll(x)); x &= x - 1; }
        }
        for (int a : nb) {
            uint64_t* ra = &G[(size_t)a * W];
            const uint64_t* rv = &G[(size_t)v * W];
            for (int w = 0; w < W; ++w) ra[w] |= rv[w];
            ra[a / 64] &= ~(1ull << (a % 64));
            ra[v / 64] &= ~(1ull << (v % 64));
            deg[a] = popc(a);
        }
        alive[v] = 0;
    }
    *flops = fl;
    *nnz = nz;
}

void compute_layout(const Tables& t, Layout& L) {
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + std::max<size_t>(bytes, 1)); return o; };
    const size_t nc = (size_t)t.n_cells;
    L.coef = take(4 * nc * sizeof(double));
    L.scale = take(nc * sizeof(double));
    L.scf = take(nc * sizeof(float));
    L.tsc = take(nc * sizeof(float));
    L.rhs_part = take(nc * sizeof(double));
    L.face_tr = take(t.faces.size() * sizeof(double));
    L.face_beta = take(t.faces.size() * sizeof(double));
    L.face_u = take(t.faces.size() * sizeof(double));
    L.face_bst = take(t.faces.size() * sizeof(double));
    L.W = take((size_t)t.total_w * (t.cfg.precision == MRCM_FP64 ? sizeof(double) : sizeof(float)));
    L.X = take((size_t)t.total_x * sizeof(double));
    L.R = take(t.cfg.precision == MRCM_FP64 ? (size_t)t.total_x * sizeof(double) : (size_t)t.total_x * sizeof(float));
    L.colnorm = take((size_t)t.total_rhs * 2 * sizeof(double));
    L.conv = take((size_t)t.total_rhs * sizeof(int));
    L.elem = take((size_t)t.total_el * sizeof(double));
    L.elem_b = take((size_t)t.total_elb * sizeof(double));
    L.csr_val = take(t.colidx.size() * sizeof(double));
    L.b_int = take((size_t)2 * t.NV * sizeof(double));
    L.dscale = take((size_t)2 * t.NV * sizeof(double));
    L.fronts = take((size_t)t.total_front * sizeof(double));
    L.frhs = take((size_t)t.total_frhs * sizeof(double));
    L.panel = take((size_t)t.total_panels * 32 * 32 * sizeof(double));
    L.oz = take((size_t)t.oz_rows * 1024);                 // 2 operands x 8 slices x 32 bf16 per row
    L.oz_exp = take((size_t)t.oz_rows * 2 * sizeof(int));
    L.xres = take((size_t)2 * t.NV * sizeof(double));
    L.xtmp = take((size_t)2 * t.NV * sizeof(double));
    L.psum = take(((size_t)t.subs.size() + 64) * sizeof(double));
    L.status = take(ST_COUNT * sizeof(int));
    {
        size_t parts, cnts;
        bwd_split_sizes(t.levels, t.fronts, &parts, &cnts);
        L.bpart = take(parts * sizeof(double));
        L.bcnt = take(cnts * sizeof(unsigned));
    }
    {
        int cap;
        long long stride, ystride;
        fallback_params(t, &cap, &stride, &ystride);
        L.fb_W = take((size_t)cap * stride * sizeof(double));
        L.fb_Y = take((size_t)cap * ystride * sizeof(double));
        L.fb_subs = take((size_t)cap * sizeof(SubInfo));
        L.fb_list = take((size_t)cap * sizeof(int));
    }
    L.pp_list = take((size_t)std::max<size_t>(t.subs.size(), 1) * sizeof(int));
    L.big = take((size_t)t.big_slots * ((size_t)kMaxBlock * (kMaxBlock + 1) / 2) * sizeof(double));
    L.total = off;
}

}  // namespace mrcm
