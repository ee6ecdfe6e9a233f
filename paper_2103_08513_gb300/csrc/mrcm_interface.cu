// Interface system of libmrcm (Eq. interface_problem): deterministic
// assembly of A^int from the per-subdomain blocks, and its FP64 solution by a
// nested-dissection multifrontal LDL^T.
//
// Assembly.  Basis phi_i lives on one interface Gamma_{l,l'}, so row i of
// A^int receives exactly the two subdomain blocks of l and l'; every CSR
// entry is the sum (lower side first) of at most two block entries, which
// makes the gather deterministic without atomics.
//
// Structure used by the solver.  From the Robin-to-flux map of each
// subdomain, M_l = T_R E A_l^{-1} E^T T_R - T_R (symmetric, -T_R <= M_l <= 0):
//   A^PP = sum R^T M R            symmetric negative semi-definite, null
//                                 vector "all pi^p equal" when no wall is
//                                 Dirichlet (the pressure constant);
//   A^UU = -sum R^T (beta M beta + beta A_f) R   symmetric negative definite
//                                 (beta M beta + beta A_f >= beta A_f h/(2K)/(h/(2K)+beta) > 0);
//   A^UP = -(A^PU)^T.
// Hence K = J A^int with J = diag(I, -I) is symmetric, and after adding
// -delta e_0 e_0^T to A^int (delta = |A_00|, which leaves the solution with
// pi^p_0 = 0 unchanged when b^int is consistent) it is symmetric
// quasi-definite: [[-E, F], [F^T, G]] with E, G positive definite.  Such
// matrices have an LDL^T factorisation for every symmetric ordering, so the
// fronts are factored without pivoting.  The system is also scaled
// symmetrically, K^ = D K D with D = diag(|a_ii|^{-1/2}).
//
// Elimination tree.  The subdomain grid is bisected recursively (longest axis
// first).  A node's front holds the dofs of the interfaces between its two
// halves (eliminated there, "E") and the dofs still coupled to the outside
// ("B").  Fronts are dense FP64 (lower triangle used), assembled by
// extend-add of the two children (subdomain blocks at the leaves), partially
// factored by a blocked right-looking LDL^T (32-column panels, 64x64 update
// tiles spread over the whole GPU), and leave the Schur complement on B for
// their parent.  The solution is refined once in FP64 with CSR residuals.
#include <cuda_runtime.h>

#include <algorithm>

#include "mrcm_internal.h"

namespace mrcm {

namespace {

constexpr int kThreads = 256;
constexpr int kPanel = 32;        // LDL^T panel width
constexpr int kRowTile = 256;     // rows per panel-solve CTA
constexpr int kTile = 64;         // trailing-update and assembly tile
constexpr int kRefine = 1;        // FP64 refinement steps of the interface solve

__global__ void k_assemble_csr(int nrows, const int* __restrict__ rowptr, const long long* __restrict__ src_lo,
                               const long long* __restrict__ src_hi, const int* __restrict__ rsl,
                               const int* __restrict__ rsh, const int* __restrict__ colidx,
                               const double* __restrict__ elem, const double* __restrict__ elem_b,
                               double* __restrict__ val, double* __restrict__ b, double* __restrict__ dscale) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    double diag = 0.0;
    for (int q = rowptr[r]; q < rowptr[r + 1]; ++q) {
        double v = 0.0;
        if (src_lo[q] >= 0) v += elem[src_lo[q]];
        if (src_hi[q] >= 0) v += elem[src_hi[q]];
        val[q] = v;
        if (colidx[q] == r) diag = v;
    }
    b[r] = elem_b[rsl[r]] + elem_b[rsh[r]];
    double ad = fabs(diag);
    dscale[r] = ad > 0.0 ? rsqrt(ad) : 1.0;
}

__device__ __forceinline__ double dof_sign(int dof, int NV) { return dof < NV ? 1.0 : -1.0; }

// Front assembly as a gather: every lower-triangle entry (r >= q) of the
// front is written once, as the sum (child 0 first) of the children's
// entries at the same dofs -- J-signed, scaled subdomain blocks for leaves,
// the lower triangle of the Schur complement otherwise.  64x64 tiles of the
// lower triangle are spread over the grid; blockIdx.y selects the front.
__global__ void __launch_bounds__(kThreads)
k_front_assemble(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids,
                 const int* __restrict__ inv, const int* __restrict__ dofs, const SubInfo* __restrict__ subs,
                 const double* __restrict__ elem, const double* __restrict__ dscale, int NV,
                 double* __restrict__ F) {
    const FrontInfo fr = fronts[ids[blockIdx.y]];
    const int n = fr.n;
    const int nt = (n + kTile - 1) / kTile;
    const int t = blockIdx.x;
    if (t >= nt * (nt + 1) / 2) return;
    int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    const int tj = t - ti * (ti + 1) / 2;
    double* Fm = F + fr.f_off;
    const int* fd = dofs + fr.e_dof_off;
    const int* inv0 = inv + fr.inv_off;
    const int* inv1 = inv0 + n;
    const double* src[2];
    int ld[2], off[2];
    bool leaf[2];
    for (int ci = 0; ci < 2; ++ci) {
        const int c = fr.child[ci];
        leaf[ci] = c < 0;
        if (c < 0) {
            const SubInfo& s = subs[-(c + 1)];
            src[ci] = elem + s.el_off;
            ld[ci] = s.el_dim;
            off[ci] = 0;
        } else {
            const FrontInfo& cf = fronts[c];
            src[ci] = F + cf.f_off;
            ld[ci] = cf.n;
            off[ci] = cf.ne;
        }
    }
    for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
        const int r = ti * kTile + e / kTile;
        const int q = tj * kTile + e % kTile;
        if (r >= n || q > r) continue;
        double v = 0.0;
        const int dr = fd[r], dq = fd[q];
#pragma unroll
        for (int ci = 0; ci < 2; ++ci) {
            const int* iv = ci == 0 ? inv0 : inv1;
            const int ir = iv[r], iq = iv[q];
            if (ir < 0 || iq < 0) continue;
            if (leaf[ci]) {
                v += dof_sign(dr, NV) * src[ci][(long long)ir * ld[ci] + iq] * dscale[dr] * dscale[dq];
            } else {
                const int a = off[ci] + max(ir, iq), b2 = off[ci] + min(ir, iq);
                v += src[ci][(long long)a * ld[ci] + b2];
            }
        }
        if (r == fr.pin_row && q == fr.pin_row) v -= 1.0;
        Fm[(long long)r * n + q] = v;
    }
}

// Panel step of the blocked LDL^T: every CTA factors the diagonal block
// [k0, k0+nbk) of its front in shared memory (redundantly: the factored
// block must not be written to the front while other CTAs of the same launch
// still read it), then solves its tile of rows below, l = f L11^{-T} D^{-1},
// one thread per row.  CTA x = 0 leaves the factored block (L11 strict lower,
// D on the diagonal) in `scratch`; the trailing-update kernel copies it into
// the front.
__global__ void __launch_bounds__(kThreads)
k_ldl_panel(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids, int k0,
            const double* __restrict__ F, double* __restrict__ Fw, double* __restrict__ scratch,
            int* __restrict__ status) {
    const FrontInfo fr = fronts[ids[blockIdx.y]];
    if (k0 >= fr.ne) return;
    const int n = fr.n;
    const int nbk = min(kPanel, fr.ne - k0);
    const int r0 = k0 + nbk + blockIdx.x * kRowTile;
    if (blockIdx.x > 0 && r0 >= n) return;
    const double* A = F + fr.f_off;
    __shared__ double L[kPanel][kPanel + 1];
    __shared__ double Dinv[kPanel];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // 32 x 8
    for (int i = ty; i < kPanel; i += 8) L[i][tx] = (i < nbk && tx <= i) ? A[(long long)(k0 + i) * n + k0 + tx] : 0.0;
    __syncthreads();
    int zero = 0;
    for (int k = 0; k < nbk; ++k) {
        if (threadIdx.x == 0) {
            double d = L[k][k];
            if (d == 0.0 || d != d) { zero = 1; d = 1.0; L[k][k] = 1.0; }
            Dinv[k] = 1.0 / d;
        }
        __syncthreads();
        const double inv = Dinv[k];
        // l_ik for i > k (column k scaled in place after the trailing update below)
        for (int i = k + 1 + ty; i < nbk; i += 8) {
            const double lik = L[i][k] * inv;
            for (int j = k + 1 + tx; j <= i; j += 32) L[i][j] -= lik * L[j][k];
        }
        __syncthreads();
        if (threadIdx.x < 32 && k + 1 + tx < nbk) L[k + 1 + tx][k] *= inv;
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        double* sc = scratch + (long long)blockIdx.y * kPanel * kPanel;
        for (int i = ty; i < nbk; i += 8) sc[i * kPanel + tx] = (tx <= i) ? L[i][tx] : 0.0;
        if (zero && threadIdx.x == 0) atomicAdd(&status[ST_ZERO_PIVOT], 1);
    }
    const int r = r0 + threadIdx.x;
    if (r < n) {
        double* row = Fw + fr.f_off + (long long)r * n + k0;
        double w[kPanel];
#pragma unroll
        for (int j = 0; j < kPanel; ++j) w[j] = j < nbk ? row[j] : 0.0;
#pragma unroll
        for (int j = 0; j < kPanel; ++j) {
            double acc = w[j];
#pragma unroll
            for (int k = 0; k < j; ++k) acc -= w[k] * L[j][k];
            w[j] = acc;
        }
#pragma unroll
        for (int j = 0; j < kPanel; ++j)
            if (j < nbk) row[j] = w[j] * Dinv[j];
    }
}

// Trailing update of the blocked LDL^T: F22 -= L21 D L21^T on 64x64 tiles of
// the lower triangle; blockIdx.x enumerates the (ti >= tj) tile pairs.
__global__ void __launch_bounds__(kThreads)
k_ldl_update(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids, int k0, double* __restrict__ F,
             const double* __restrict__ scratch) {
    const FrontInfo fr = fronts[ids[blockIdx.y]];
    if (k0 >= fr.ne) return;
    const int n = fr.n;
    const int nbk = min(kPanel, fr.ne - k0);
    const int k1 = k0 + nbk;
    const int m = n - k1;
    if (blockIdx.x == 0) {                  // commit the factored diagonal block of this panel
        const double* sc = scratch + (long long)blockIdx.y * kPanel * kPanel;
        double* A0 = F + fr.f_off;
        for (int e = threadIdx.x; e < kPanel * kPanel; e += blockDim.x) {
            const int i = e >> 5, j = e & 31;
            if (i < nbk && j <= i) A0[(long long)(k0 + i) * n + k0 + j] = sc[e];
        }
    }
    if (m <= 0) return;
    const int nt = (m + kTile - 1) / kTile;
    const int T = nt * (nt + 1) / 2;
    const int t = blockIdx.x;
    if (t >= T) return;
    int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    const int tj = t - ti * (ti + 1) / 2;
    double* A = F + fr.f_off;
    __shared__ double Li[kTile][kPanel + 1];
    __shared__ double Lj[kTile][kPanel + 1];
    __shared__ double Dk[kPanel];
    {
        const double* sc = scratch + (long long)blockIdx.y * kPanel * kPanel;
        for (int k = threadIdx.x; k < kPanel; k += blockDim.x) Dk[k] = k < nbk ? sc[k * kPanel + k] : 0.0;
    }
    __syncthreads();
    const int i0 = k1 + ti * kTile, j0 = k1 + tj * kTile;
    for (int e = threadIdx.x; e < kTile * kPanel; e += blockDim.x) {
        int a = e / kPanel, k = e % kPanel;
        int gi = i0 + a, gj = j0 + a;
        Li[a][k] = (gi < n && k < nbk) ? A[(long long)gi * n + k0 + k] * Dk[k] : 0.0;
        Lj[a][k] = (gj < n && k < nbk) ? A[(long long)gj * n + k0 + k] : 0.0;
    }
    __syncthreads();
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    double acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;
    for (int k = 0; k < nbk; ++k) {
        double a[4], bb[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) a[p] = Li[ty + 16 * p][k];
#pragma unroll
        for (int q = 0; q < 4; ++q) bb[q] = Lj[tx + 16 * q][k];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * bb[q];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        int gi = i0 + ty + 16 * p;
        if (gi >= n) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int gj = j0 + tx + 16 * q;
            if (gj < n && gj <= gi) A[(long long)gi * n + gj] -= acc[p][q];
        }
    }
}

// Forward substitution of one front: r = children's reduced rhs + the scaled,
// J-signed global rhs of its E dofs; then L y = r over the E columns.  y_E is
// divided by D; the reduced B part stays in frhs for the parent.
__global__ void __launch_bounds__(kThreads)
k_front_forward(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids,
                const int* __restrict__ maps, const int* __restrict__ dofs,
                const double* __restrict__ F, const double* __restrict__ bglob,
                const double* __restrict__ dscale, int NV, double* __restrict__ frhs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* r = reinterpret_cast<double*>(smem_raw);
    const FrontInfo fr = fronts[ids[blockIdx.x]];
    const int n = fr.n, ne = fr.ne;
    const double* A = F + fr.f_off;
    const int* fd = dofs + fr.e_dof_off;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        double v = 0.0;
        if (q < ne) { int d = fd[q]; v = dof_sign(d, NV) * dscale[d] * bglob[d]; }
        r[q] = v;
    }
    __syncthreads();
    for (int ci = 0; ci < 2; ++ci) {
        const int c = fr.child[ci];
        if (c < 0) continue;
        const FrontInfo cf = fronts[c];
        const int* mp = maps + fr.map_off[ci];
        for (int q = threadIdx.x; q < cf.nb; q += blockDim.x) r[mp[q]] += frhs[cf.r_off + cf.ne + q];
        __syncthreads();
    }
    for (int k0 = 0; k0 < ne; k0 += kPanel) {
        const int k1 = min(ne, k0 + kPanel);
        if (threadIdx.x < 32) {
            for (int k = k0; k < k1; ++k) {
                double rk = r[k];
                __syncwarp();
                int i = k + 1 + threadIdx.x;
                if (i < k1) r[i] -= A[(long long)i * n + k] * rk;
                __syncwarp();
            }
        }
        __syncthreads();
        for (int i = k1 + threadIdx.x; i < n; i += blockDim.x) {
            double acc = r[i];
            const double* row = A + (long long)i * n;
            for (int k = k0; k < k1; ++k) acc -= row[k] * r[k];
            r[i] = acc;
        }
        __syncthreads();
    }
    double* out = frhs + fr.r_off;
    for (int q = threadIdx.x; q < n; q += blockDim.x) out[q] = q < ne ? r[q] / A[(long long)q * n + q] : r[q];
}

// Backward substitution of one front: x_B (scaled) from the ancestors, then
// L_EE^T x_E = z_E - L_BE^T x_B.
__global__ void __launch_bounds__(kThreads)
k_front_backward(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids,
                 const int* __restrict__ dofs, const double* __restrict__ F,
                 const double* __restrict__ frhs, double* __restrict__ xs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* w = reinterpret_cast<double*>(smem_raw);
    const FrontInfo fr = fronts[ids[blockIdx.x]];
    const int n = fr.n, ne = fr.ne;
    const double* A = F + fr.f_off;
    const int* fd = dofs + fr.e_dof_off;
    for (int i = threadIdx.x; i < ne; i += blockDim.x) {
        double acc = frhs[fr.r_off + i];
        for (int j = ne; j < n; ++j) acc -= A[(long long)j * n + i] * xs[fd[j]];
        w[i] = acc;
    }
    __syncthreads();
    const int nblk = (ne + kPanel - 1) / kPanel;
    for (int bk = nblk - 1; bk >= 0; --bk) {
        const int k0 = bk * kPanel, k1 = min(ne, k0 + kPanel);
        if (threadIdx.x < 32) {
            for (int k = k1 - 1; k >= k0; --k) {
                double xk = w[k];
                __syncwarp();
                int i = k0 + threadIdx.x;
                if (i < k) w[i] -= A[(long long)k * n + i] * xk;
                __syncwarp();
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < k0; i += blockDim.x) {
            double acc = w[i];
            for (int k = k0; k < k1; ++k) acc -= A[(long long)k * n + i] * w[k];
            w[i] = acc;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < ne; i += blockDim.x) xs[fd[i]] = w[i];
}

// r = b - (A^int - delta e0 e0^T) x   (CSR, FP64; delta = 1/d_0^2 when pinned)
__global__ void k_csr_residual(int nrows, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                               const double* __restrict__ val, const double* __restrict__ b,
                               const double* __restrict__ x, const double* __restrict__ dscale, int pin,
                               double* __restrict__ r) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    double acc = b[i];
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) acc -= val[q] * x[colidx[q]];
    if (pin && i == 0) acc += x[0] / (dscale[0] * dscale[0]);
    r[i] = acc;
}

__global__ void k_unscale(int n, const double* __restrict__ xs, const double* __restrict__ dscale,
                          double* __restrict__ x, int accumulate) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = xs[i] * dscale[i];
    x[i] = accumulate ? x[i] + v : v;
}

struct LevelPlan { int steps; std::vector<int> row_tiles, upd_tiles; };

LevelPlan plan_level(const Tables& t, int h) {
    LevelPlan p;
    int max_ne = 0;
    for (int id : t.levels[h]) max_ne = std::max(max_ne, t.fronts[id].ne);
    p.steps = (max_ne + kPanel - 1) / kPanel;
    for (int s = 0; s < p.steps; ++s) {
        int k0 = s * kPanel, rt = 1, ut = 0;
        for (int id : t.levels[h]) {
            const FrontInfo& f = t.fronts[id];
            if (k0 >= f.ne) continue;
            int k1 = k0 + std::min(kPanel, f.ne - k0);
            int m = f.n - k1;
            rt = std::max(rt, (m + kRowTile - 1) / kRowTile);
            int nt = (m + kTile - 1) / kTile;
            ut = std::max(ut, nt * (nt + 1) / 2);
        }
        p.row_tiles.push_back(rt);
        p.upd_tiles.push_back(ut);
    }
    return p;
}

}  // namespace

int launch_assemble_interface(const Tables& t, const DeviceTables& d, const Layout& L, char* ws, void* stream, Prof& P) {
    cudaStream_t st = (cudaStream_t)stream;
    const int nd = 2 * t.NV;
    if (nd == 0) return 0;
    double* dscale = (double*)(ws + L.dscale);
    MRCM_LAUNCH(P, "k_assemble_csr", st, k_assemble_csr<<<(nd + 127) / 128, 128, 0, st>>>(nd, d.rowptr, d.src_lo, d.src_hi, d.rhs_src_lo, d.rhs_src_hi,
                                                   d.colidx, (const double*)(ws + L.elem),
                                                   (const double*)(ws + L.elem_b), (double*)(ws + L.csr_val),
                                                   (double*)(ws + L.b_int), dscale));
    // numeric multifrontal factorisation, leaves to root
    double* F = (double*)(ws + L.fronts);
    double* scratch = (double*)(ws + L.panel);
    int* status = (int*)(ws + L.status);
    for (size_t h = 1; h < t.levels.size(); ++h) {
        int cnt = (int)t.levels[h].size();
        if (!cnt) continue;
        const int* ids = d.level_ids + d.level_off[h];
        int maxT = 1;
        for (int id : t.levels[h]) { int nt = (t.fronts[id].n + kTile - 1) / kTile; maxT = std::max(maxT, nt * (nt + 1) / 2); }
        dim3 ga(maxT, cnt);
        MRCM_LAUNCH(P, "k_front_assemble", st, k_front_assemble<<<ga, kThreads, 0, st>>>(d.fronts, ids, d.front_inv, d.front_dofs, d.subs,
                                                  (const double*)(ws + L.elem), dscale, t.NV, F));
        LevelPlan p = plan_level(t, (int)h);
        for (int s = 0; s < p.steps; ++s) {
            dim3 gp(p.row_tiles[s], cnt);
            MRCM_LAUNCH(P, "k_ldl_panel", st, k_ldl_panel<<<gp, kThreads, 0, st>>>(d.fronts, ids, s * kPanel, F, F,
                                                                                 scratch, status));
            dim3 gu(std::max(1, p.upd_tiles[s]), cnt);
            MRCM_LAUNCH(P, "k_ldl_update", st, k_ldl_update<<<gu, kThreads, 0, st>>>(d.fronts, ids, s * kPanel, F, scratch));
        }
    }
    return (int)cudaGetLastError();
}

static void multifrontal_solve(const Tables& t, const DeviceTables& d, const Layout& L, char* ws,
                               const double* rhs, double* xs, cudaStream_t st, Prof& P) {
    double* F = (double*)(ws + L.fronts);
    double* frhs = (double*)(ws + L.frhs);
    const double* dscale = (const double*)(ws + L.dscale);
    size_t sm = sizeof(double) * (size_t)std::max(t.max_front, 1);
    for (size_t h = 1; h < t.levels.size(); ++h) {
        int cnt = (int)t.levels[h].size();
        if (!cnt) continue;
        MRCM_LAUNCH(P, "k_front_forward", st, k_front_forward<<<cnt, kThreads, sm, st>>>(d.fronts, d.level_ids + d.level_off[h], d.front_maps,
                                                  d.front_dofs, F, rhs, dscale, t.NV, frhs));
    }
    for (size_t h = t.levels.size() - 1; h >= 1; --h) {
        int cnt = (int)t.levels[h].size();
        if (!cnt) continue;
        MRCM_LAUNCH(P, "k_front_backward", st, k_front_backward<<<cnt, kThreads, sm, st>>>(d.fronts, d.level_ids + d.level_off[h], d.front_dofs, F,
                                                   frhs, xs));
    }
}

int configure_interface(const Tables& t, DeviceTables& d) {
    d.front_smem = sizeof(double) * (size_t)std::max(t.max_front, 1);
    if (d.front_smem > 48 * 1024) {
        cudaFuncSetAttribute(k_front_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.front_smem);
        cudaFuncSetAttribute(k_front_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.front_smem);
    }
    return (int)cudaGetLastError();
}

int launch_solve_interface(const Tables& t, const DeviceTables& d, const Layout& L, char* ws, double* X,
                           void* stream, Prof& P) {
    cudaStream_t st = (cudaStream_t)stream;
    const int nd = 2 * t.NV;
    if (nd == 0) return 0;
    const double* b = (const double*)(ws + L.b_int);
    const double* dscale = (const double*)(ws + L.dscale);
    double* r = (double*)(ws + L.xres);
    double* xs = (double*)(ws + L.xtmp);
    const int pin = t.has_dirichlet ? 0 : 1;
    multifrontal_solve(t, d, L, ws, b, xs, st, P);
    MRCM_LAUNCH(P, "k_unscale", st, k_unscale<<<(nd + 255) / 256, 256, 0, st>>>(nd, xs, dscale, X, 0));
    for (int it = 0; it < kRefine; ++it) {
        MRCM_LAUNCH(P, "k_csr_residual", st, k_csr_residual<<<(nd + 127) / 128, 128, 0, st>>>(nd, d.rowptr, d.colidx, (const double*)(ws + L.csr_val),
                                                       b, X, dscale, pin, r));
        multifrontal_solve(t, d, L, ws, r, xs, st, P);
        MRCM_LAUNCH(P, "k_unscale", st, k_unscale<<<(nd + 255) / 256, 256, 0, st>>>(nd, xs, dscale, X, 1));
    }
    return (int)cudaGetLastError();
}

}  // namespace mrcm
