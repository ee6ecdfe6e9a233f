// Local subdomain kernels of libmrcm: TPFA + Robin assembly, slab block
// factorisation, multi-RHS block solves, FP64 residuals and the reduction of
// MBF flux traces to per-subdomain interface blocks.
//
// Local problem (Eq. localomegapar, Eq. localomegaint discretised as in
// Eq. darcy-discrete / Eq. aijk, times the cell volume): for every cell c of
// subdomain l
//   sum_{interior faces} T (p_c - p_nb) + sum_{Robin faces} T_R (p_c - g_f)
//     + sum_{Dirichlet walls} T_D (p_c - g_D) = f_c V
// with T = A_f * 2 K_a K_b / (K_a + K_b) / h_n, T_R = A_f / (h_n/(2 K_n) + beta)
// and T_D = 2 K_n A_f / h_n.
//
// Storage: cells are numbered slab-major (see SubInfo), which makes A^H_l
// block tridiagonal, A = tridiag(-diag(t_{s-1}), D_s, -diag(t_s)), D_s the
// in-slab 5-point blocks.  The factor kept is W_s = S_s^{-1}, the inverses of
// the block pivots of the block LU recursion
//   S_0 = D_0,  S_s = D_s - diag(t_{s-1}) W_{s-1} diag(t_{s-1}),
// so that both sweeps of a solve are small dense products W_s * Z.
//
// Mixed precision: the factor and the sweeps run on the Jacobi-scaled matrix
// A^ = S A S, S = diag(1/sqrt(a_cc)), in FP32; FP64 residuals of the unscaled
// matrix drive iterative refinement.
#include <cuda_runtime.h>

#include <cstdint>

#include "mrcm_internal.h"

namespace mrcm {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double harm(double a, double b) { return 2.0 * a * b / (a + b); }

struct Geo {
    double h[3];
    double area[3];
    int n[3];
};

__device__ __forceinline__ void local_coords(const SubInfo& s, int c, int lc[3]) {
    int sl = c / s.b;
    int r = c - sl * s.b;
    int v = r / s.su;
    int u = r - v * s.su;
    lc[s.sa] = sl;
    lc[s.ua] = u;
    lc[s.va] = v;
}

__device__ __forceinline__ long long global_cell(const SubInfo& s, const int lc[3], const int n[3]) {
    return (long long)(s.o[0] + lc[0]) + (long long)n[0] * ((s.o[1] + lc[1]) + (long long)n[1] * (s.o[2] + lc[2]));
}

__device__ __forceinline__ double beta_of(int mode, double alpha, double beta_const, const SubInfo& s,
                                          int a, double h_a, double Kn) {
    return mode == MRCM_BETA_CONST ? beta_const : alpha * (double)s.sz[a] * h_a / Kn;
}

// ---------------------------------------------------------------------------
// Per-cell coefficients (FP64): diagonal (incl. Robin and Dirichlet terms),
// the three "+" transmissibilities along (u, v, s), the Jacobi scale and the
// Dirichlet part of the particular right-hand side.  Also T_R and beta of
// every Robin face.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_coefficients(const SubInfo* __restrict__ subs, const FaceInfo* __restrict__ faces,
               const double* __restrict__ K, Geo geo, int beta_mode, double alpha, double beta_const,
               int4 bc_lo_hi /* x: mask of Dirichlet low walls, y: high walls */,
               double3 bc_lo, double3 bc_hi,
               double* __restrict__ coef, double* __restrict__ scale, double* __restrict__ rhs_dir,
               double* __restrict__ face_tr, double* __restrict__ face_beta, long long ncell_total) {
    const SubInfo s = subs[blockIdx.x];
    const long long ncells = (long long)geo.n[0] * geo.n[1] * geo.n[2];
    const double* Kc[3] = {K, K + ncells, K + 2 * ncells};
    const long long stride[3] = {1, geo.n[0], (long long)geo.n[0] * geo.n[1]};
    const double blo[3] = {bc_lo.x, bc_lo.y, bc_lo.z};
    const double bhi[3] = {bc_hi.x, bc_hi.y, bc_hi.z};
    for (int c = threadIdx.x; c < s.N; c += blockDim.x) {
        int lc[3];
        local_coords(s, c, lc);
        long long g = global_cell(s, lc, geo.n);
        double d = 0.0, tplus[3] = {0.0, 0.0, 0.0}, rd = 0.0;
        for (int a = 0; a < 3; ++a) {
            double ka = Kc[a][g];
            // +a side
            if (lc[a] + 1 < s.sz[a]) {
                double T = geo.area[a] * harm(ka, Kc[a][g + stride[a]]) / geo.h[a];
                tplus[a] = T;
                d += T;
            } else if (s.o[a] + lc[a] == geo.n[a] - 1) {
                if ((bc_lo_hi.y >> a) & 1) { double TD = geo.area[a] * 2.0 * ka / geo.h[a]; d += TD; rd += TD * bhi[a]; }
            } else {
                double beta = beta_of(beta_mode, alpha, beta_const, s, a, geo.h[a], ka);
                d += geo.area[a] / (geo.h[a] / (2.0 * ka) + beta);
            }
            // -a side
            if (lc[a] > 0) {
                d += geo.area[a] * harm(ka, Kc[a][g - stride[a]]) / geo.h[a];
            } else if (s.o[a] == 0) {
                if ((bc_lo_hi.x >> a) & 1) { double TD = geo.area[a] * 2.0 * ka / geo.h[a]; d += TD; rd += TD * blo[a]; }
            } else {
                double beta = beta_of(beta_mode, alpha, beta_const, s, a, geo.h[a], ka);
                d += geo.area[a] / (geo.h[a] / (2.0 * ka) + beta);
            }
        }
        long long i = s.cell_off + c;
        coef[i] = d;
        coef[ncell_total + i] = tplus[s.ua];
        coef[2 * ncell_total + i] = tplus[s.va];
        coef[3 * ncell_total + i] = tplus[s.sa];
        scale[i] = rsqrt(d);
        rhs_dir[i] = rd;
    }
    for (int q = threadIdx.x; q < s.nface; q += blockDim.x) {
        FaceInfo fi = faces[s.face_off + q];
        int lc[3];
        local_coords(s, fi.cell, lc);
        long long g = global_cell(s, lc, geo.n);
        int a = fi.axis;
        double ka = Kc[a][g];
        double beta = beta_of(beta_mode, alpha, beta_const, s, a, geo.h[a], ka);
        face_tr[s.face_off + q] = geo.area[a] / (geo.h[a] / (2.0 * ka) + beta);
        face_beta[s.face_off + q] = beta;
    }
}

// ---------------------------------------------------------------------------
// Slab block factorisation: W_s = S_s^{-1} by in-place Gauss-Jordan on the
// SPD block pivot (no pivoting needed for SPD).  One CTA per subdomain; the
// running block lives in shared memory.
// ---------------------------------------------------------------------------
template <typename T, bool kScaled>
__global__ void __launch_bounds__(kThreads)
k_block_factor(const SubInfo* __restrict__ subs, const double* __restrict__ coef,
               const double* __restrict__ scale, T* __restrict__ Wall, int* __restrict__ status,
               long long nct, int bmax) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* A = reinterpret_cast<T*>(smem_raw);          // b x b, row major
    T* col = A + bmax * bmax;                        // pivot column
    T* row = col + bmax;                             // pivot row
    const SubInfo s = subs[blockIdx.x];
    const int b = s.b, su = s.su;
    const double* cd = coef + s.cell_off;
    const double* cu = coef + nct + s.cell_off;
    const double* cv = coef + 2 * nct + s.cell_off;
    const double* cs = coef + 3 * nct + s.cell_off;
    const double* sc = scale + s.cell_off;
    T* W = Wall + s.w_off;
    int bad = 0;
    for (int sl = 0; sl < s.ns; ++sl) {
        const int base = sl * b;
        // S_s = D_s - diag(t) W_{s-1} diag(t), in place over W_{s-1}
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
            int i = e / b, j = e - (e / b) * b;
            double dij = 0.0;
            int ci = base + i, cj = base + j;
            if (i == j) dij = cd[ci];
            else {
                int ui = i % su, uj = j % su;
                if (j == i + 1 && uj == ui + 1) dij = -cu[ci];
                else if (i == j + 1 && ui == uj + 1) dij = -cu[cj];
                else if (j == i + su) dij = -cv[ci];
                else if (i == j + su) dij = -cv[cj];
            }
            if (kScaled) dij *= sc[ci] * sc[cj];
            double v = dij;
            if (sl > 0) {
                double ti = cs[ci - b], tj = cs[cj - b];
                if (kScaled) { ti *= sc[ci - b] * sc[ci]; tj *= sc[cj - b] * sc[cj]; }
                v -= ti * tj * (double)A[e];
            }
            A[e] = (T)v;
        }
        __syncthreads();
        // in-place Gauss-Jordan inversion (row k and column k saved separately:
        // the intermediate matrices are not symmetric)
        for (int k = 0; k < b; ++k) {
            T p = A[k * b + k];
            for (int i = threadIdx.x; i < b; i += blockDim.x) { col[i] = A[i * b + k]; row[i] = A[k * b + i]; }
            __syncthreads();
            if (!(p > (T)0)) { bad = 1; p = (T)1; }
            T ip = (T)1 / p;
            for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
                int i = e / b, j = e - (e / b) * b;
                T v;
                if (i == k && j == k) v = ip;
                else if (i == k) v = row[j] * ip;
                else if (j == k) v = -col[i] * ip;
                else v = A[e] - col[i] * row[j] * ip;
                A[e] = v;
            }
            __syncthreads();
        }
        // W_s: the block is symmetric; store it
        T* Ws = W + (long long)sl * b * b;
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) Ws[e] = A[e];
        __syncthreads();
    }
    if (bad && threadIdx.x == 0) atomicAdd(&status[ST_NOT_SPD], 1);
}

// ---------------------------------------------------------------------------
// Right-hand sides of all MBFs and the particular problem, written in place
// into the MBF array [m][N] of each subdomain:
//   P-MBF k: T_R on the faces of basis k;  U-MBF k: -beta s T_R on them;
//   particular: f V + Dirichlet wall terms.
// Each (cell, column) is written by at most one face: a cell has one face
// per side and a basis lives on one side of one interface.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_rhs(const SubInfo* __restrict__ subs, const FaceInfo* __restrict__ faces,
      const double* __restrict__ face_tr, const double* __restrict__ face_beta,
      const double* __restrict__ rhs_dir, const double* __restrict__ f, Geo geo,
      double* __restrict__ X) {
    const SubInfo s = subs[blockIdx.x];
    double* Xs = X + s.x_off;
    const double vol = geo.h[0] * geo.h[1] * geo.h[2];
    const long long nN = (long long)s.m * s.N;
    for (long long e = threadIdx.x; e < nN - s.N; e += blockDim.x) Xs[e] = 0.0;
    double* part = Xs + (long long)(s.m - 1) * s.N;
    for (int c = threadIdx.x; c < s.N; c += blockDim.x) {
        int lc[3];
        local_coords(s, c, lc);
        part[c] = rhs_dir[s.cell_off + c] + f[global_cell(s, lc, geo.n)] * vol;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < s.nface; q += blockDim.x) {
        FaceInfo fi = faces[s.face_off + q];
        double tr = face_tr[s.face_off + q];
        Xs[(long long)fi.col * s.N + fi.cell] = tr;
        Xs[(long long)(s.nI + fi.col) * s.N + fi.cell] = -face_beta[s.face_off + q] * fi.s * tr;
    }
}

// ---------------------------------------------------------------------------
// Multi-RHS block solve on one subdomain (all m columns), in place:
//   forward   Z_s = r_s + t_{s-1} o Y_{s-1},   Y_s = W_s Z_s   (Y_s overwrites r_s)
//   backward  x_s = Y_s + W_s (t_s o x_{s+1})
// The result is written to `out` (overwrite, or accumulate when kAccumulate).
// In scaled (mixed) mode the solve is for A^ = S A S: r is scaled by S on
// input and x by S on output.
// ---------------------------------------------------------------------------
constexpr int kMaxColsPerThread = 16;

template <typename T, bool kScaled, bool kAccumulate>
__global__ void __launch_bounds__(kThreads)
k_block_solve(const SubInfo* __restrict__ subs, const double* __restrict__ coef,
              const double* __restrict__ scale, const T* __restrict__ Wall,
              double* __restrict__ inout, double* __restrict__ out, long long nct,
              const int* __restrict__ skip_flag) {
    if (skip_flag && *skip_flag == 0) return;     // every column already converged
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SubInfo s = subs[blockIdx.x];
    const int b = s.b, m = s.m, N = s.N;
    T* Wsm = reinterpret_cast<T*>(smem_raw);       // b x b
    T* Z = Wsm + b * b;                            // b x m, column major (Z[j*b + i])
    T* Yp = Z + b * m;                             // previous slab's result
    const double* cs = coef + 3 * nct + s.cell_off;
    const double* sc = scale + s.cell_off;
    const T* W = Wall + s.w_off;
    double* io = inout + s.x_off;
    double* ou = out + s.x_off;
    const int groups = blockDim.x / b;             // b <= 128 so groups >= 2
    const int i = threadIdx.x % b;
    const int jg = threadIdx.x / b;
    const bool active = jg < groups;

    // ---- forward sweep
    for (int sl = 0; sl < s.ns; ++sl) {
        const int base = sl * b;
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) Wsm[e] = W[(long long)sl * b * b + e];
        for (int e = threadIdx.x; e < b * m; e += blockDim.x) {
            int j = e / b, ii = e - j * b;
            double r = io[(long long)j * N + base + ii];
            if (kScaled) r *= sc[base + ii];
            if (sl > 0) {
                double t = cs[base - b + ii];
                if (kScaled) t *= sc[base - b + ii] * sc[base + ii];
                r += t * (double)Yp[e];
            }
            Z[e] = (T)r;
        }
        __syncthreads();
        if (active) {
            for (int j0 = jg; j0 < m; j0 += groups * kMaxColsPerThread) {
                T acc[kMaxColsPerThread];
#pragma unroll
                for (int q = 0; q < kMaxColsPerThread; ++q) acc[q] = (T)0;
                for (int k = 0; k < b; ++k) {
                    T w = Wsm[k * b + i];                       // W symmetric
#pragma unroll
                    for (int q = 0; q < kMaxColsPerThread; ++q) {
                        int j = j0 + q * groups;
                        if (j < m) acc[q] += w * Z[j * b + k];
                    }
                }
#pragma unroll
                for (int q = 0; q < kMaxColsPerThread; ++q) {
                    int j = j0 + q * groups;
                    if (j < m) {
                        Yp[j * b + i] = acc[q];
                        io[(long long)j * N + base + i] = (double)acc[q];
                    }
                }
            }
        }
        __syncthreads();
    }
    // ---- backward sweep (Yp now holds x_{s+1} scratch)
    for (int sl = s.ns - 1; sl >= 0; --sl) {
        const int base = sl * b;
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) Wsm[e] = W[(long long)sl * b * b + e];
        for (int e = threadIdx.x; e < b * m; e += blockDim.x) {
            int ii = e % b;
            double v = 0.0;
            if (sl < s.ns - 1) {
                double t = cs[base + ii];
                if (kScaled) t *= sc[base + ii] * sc[base + b + ii];
                v = t * (double)Yp[e];
            }
            Z[e] = (T)v;
        }
        __syncthreads();
        if (active) {
            for (int j0 = jg; j0 < m; j0 += groups * kMaxColsPerThread) {
                T acc[kMaxColsPerThread];
#pragma unroll
                for (int q = 0; q < kMaxColsPerThread; ++q) acc[q] = (T)0;
                if (sl < s.ns - 1) {
                    for (int k = 0; k < b; ++k) {
                        T w = Wsm[k * b + i];
#pragma unroll
                        for (int q = 0; q < kMaxColsPerThread; ++q) {
                            int j = j0 + q * groups;
                            if (j < m) acc[q] += w * Z[j * b + k];
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < kMaxColsPerThread; ++q) {
                    int j = j0 + q * groups;
                    if (j < m) {
                        long long gi = (long long)j * N + base + i;
                        double x = io[gi] + (double)acc[q];      // Y_s + W_s (t o x_{s+1})
                        Yp[j * b + i] = (T)x;
                        double xo = kScaled ? x * sc[base + i] : x;
                        if (kAccumulate) ou[gi] += xo; else ou[gi] = xo;
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FP64 residual R = B - A X of every MBF column (unscaled matrix), and the
// per-subdomain count of columns with ||r||_2 > tol ||b||_2.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_residual(const SubInfo* __restrict__ subs, const FaceInfo* __restrict__ faces,
           const double* __restrict__ coef, const double* __restrict__ face_tr,
           const double* __restrict__ face_beta, const double* __restrict__ rhs_dir,
           const double* __restrict__ f, Geo geo, const double* __restrict__ X,
           double* __restrict__ R, long long nct, double tol, int* __restrict__ status) {
    const SubInfo s = subs[blockIdx.x];
    const int N = s.N, b = s.b, su = s.su, m = s.m;
    const double* cd = coef + s.cell_off;
    const double* cu = coef + nct + s.cell_off;
    const double* cv = coef + 2 * nct + s.cell_off;
    const double* cs = coef + 3 * nct + s.cell_off;
    const double* Xs = X + s.x_off;
    double* Rs = R + s.x_off;
    const double vol = geo.h[0] * geo.h[1] * geo.h[2];
    for (long long e = threadIdx.x; e < (long long)m * N; e += blockDim.x) {
        int j = (int)(e / N);
        int c = (int)(e - (long long)j * N);
        const double* x = Xs + (long long)j * N;
        int r = c % b;
        int u = r % su;
        double ax = cd[c] * x[c];
        if (u + 1 < su) ax -= cu[c] * x[c + 1];
        if (u > 0) ax -= cu[c - 1] * x[c - 1];
        if (r + su < b) ax -= cv[c] * x[c + su];
        if (r >= su) ax -= cv[c - su] * x[c - su];
        if (c + b < N) ax -= cs[c] * x[c + b];
        if (c >= b) ax -= cs[c - b] * x[c - b];
        double bval = 0.0;
        if (j == m - 1) {
            int lc[3];
            local_coords(s, c, lc);
            bval = rhs_dir[s.cell_off + c] + f[global_cell(s, lc, geo.n)] * vol;
        }
        Rs[e] = bval - ax;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < s.nface; q += blockDim.x) {
        FaceInfo fi = faces[s.face_off + q];
        double tr = face_tr[s.face_off + q];
        Rs[(long long)fi.col * N + fi.cell] += tr;
        Rs[(long long)(s.nI + fi.col) * N + fi.cell] += -face_beta[s.face_off + q] * fi.s * tr;
    }
    __syncthreads();
    // column norms: ||r_j||^2 vs ||b_j||^2 (b_j rebuilt from the faces / sources)
    __shared__ double red_r[kThreads / 32], red_b[kThreads / 32];
    __shared__ int nbad;
    if (threadIdx.x == 0) nbad = 0;
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        double rr = 0.0, bb = 0.0;
        for (int c = threadIdx.x; c < N; c += blockDim.x) { double v = Rs[(long long)j * N + c]; rr += v * v; }
        if (j < 2 * s.nI) {
            int col = j < s.nI ? j : j - s.nI;
            for (int q = threadIdx.x; q < s.nface; q += blockDim.x) {
                FaceInfo fi = faces[s.face_off + q];
                if (fi.col != col) continue;
                double tr = face_tr[s.face_off + q];
                double v = j < s.nI ? tr : face_beta[s.face_off + q] * tr;
                bb += v * v;
            }
        } else {
            for (int c = threadIdx.x; c < N; c += blockDim.x) {
                int lc[3];
                local_coords(s, c, lc);
                double v = rhs_dir[s.cell_off + c] + f[global_cell(s, lc, geo.n)] * vol;
                bb += v * v;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            rr += __shfl_down_sync(0xffffffffu, rr, o);
            bb += __shfl_down_sync(0xffffffffu, bb, o);
        }
        if ((threadIdx.x & 31) == 0) { red_r[threadIdx.x >> 5] = rr; red_b[threadIdx.x >> 5] = bb; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double tr = 0.0, tb = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tr += red_r[w]; tb += red_b[w]; }
            if (!(tr <= tol * tol * tb)) nbad += 1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && nbad) atomicAdd(&status[ST_UNCONVERGED], nbad);
}

// ---------------------------------------------------------------------------
// Flux traces q_f = T_R (p_c - g_f) of every MBF column, reduced over each
// basis' faces into the subdomain's interface block (Eq. weakcont_f and
// Eq. weakcont_p restricted to one subdomain):
//   F row k, column j:  sum_{f in phi_k} q_f[j]
//   U row k, column j:  sum_{f in phi_k} beta_f s q_f[j]   (- sum beta_f A_f on the diagonal)
//   element rhs:        -(same sums of the particular column)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_element(const SubInfo* __restrict__ subs, const FaceInfo* __restrict__ faces,
          const double* __restrict__ face_tr, const double* __restrict__ face_beta,
          const double* __restrict__ X, Geo geo, double* __restrict__ elem, double* __restrict__ elem_b) {
    const SubInfo s = subs[blockIdx.x];
    const int nI = s.nI, m = s.m, N = s.N, dim = s.el_dim;
    __shared__ int start[kMaxI + 1];                  // per-column face ranges
    for (int q = threadIdx.x; q <= nI; q += blockDim.x) start[q] = s.nface;
    __syncthreads();
    for (int q = threadIdx.x; q < s.nface; q += blockDim.x) {
        int c = faces[s.face_off + q].col;
        if (q == 0 || faces[s.face_off + q - 1].col != c) start[c] = q;
    }
    __syncthreads();
    const double* Xs = X + s.x_off;
    for (int e = threadIdx.x; e < nI * m; e += blockDim.x) {
        int k = e / m, j = e - (e / m) * m;
        int q0 = start[k], q1 = start[k + 1];
        double sf = 0.0, su = 0.0, sdiag = 0.0;
        for (int q = q0; q < q1; ++q) {
            FaceInfo fi = faces[s.face_off + q];
            double tr = face_tr[s.face_off + q], be = face_beta[s.face_off + q];
            double g = 0.0;
            if (j == fi.col) g = 1.0;
            else if (j == nI + fi.col) g = -be * fi.s;
            double qf = tr * (Xs[(long long)j * N + fi.cell] - g);
            sf += qf;
            su += be * fi.s * qf;
            sdiag += be * geo.area[fi.axis];
        }
        if (j < dim) {
            elem[s.el_off + (long long)k * dim + j] = sf;
            double uv = su;
            if (j == nI + k) uv -= sdiag;
            elem[s.el_off + (long long)(nI + k) * dim + j] = uv;
        } else {
            elem_b[s.elb_off + k] = -sf;
            elem_b[s.elb_off + nI + k] = -su;
        }
    }
}

__global__ void k_zero_int(int* p, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0;
}

__global__ void k_set_int(int* p, int v) { *p = v; }

Geo make_geo(const mrcm_config& c) {
    Geo g;
    g.h[0] = c.hx; g.h[1] = c.hy; g.h[2] = c.hz;
    g.area[0] = c.hy * c.hz; g.area[1] = c.hx * c.hz; g.area[2] = c.hx * c.hy;
    g.n[0] = c.nx; g.n[1] = c.ny; g.n[2] = c.nz;
    return g;
}

template <typename T>
size_t solve_smem(int b, int m) { return sizeof(T) * ((size_t)b * b + 2 * (size_t)b * m); }

}  // namespace

int launch_factor(const Tables& t, const DeviceTables& d, const Layout& L, char* ws,
                  const double* K, int precision, void* stream, Prof& P) {
    cudaStream_t st = (cudaStream_t)stream;
    const int nsub = (int)t.subs.size();
    const mrcm_config& c = t.cfg;
    int4 bcm = make_int4(0, 0, 0, 0);
    for (int a = 0; a < 3; ++a) {
        if (c.bc_type[a][0] == MRCM_BC_DIRICHLET) bcm.x |= 1 << a;
        if (c.bc_type[a][1] == MRCM_BC_DIRICHLET) bcm.y |= 1 << a;
    }
    double3 blo = make_double3(c.bc_value[0][0], c.bc_value[1][0], c.bc_value[2][0]);
    double3 bhi = make_double3(c.bc_value[0][1], c.bc_value[1][1], c.bc_value[2][1]);
    double* coef = (double*)(ws + L.coef);
    double* scale = (double*)(ws + L.scale);
    int* status = (int*)(ws + L.status);
    MRCM_LAUNCH(P, "k_zero_int", st, k_zero_int<<<1, 32, 0, st>>>(status, ST_COUNT));
    MRCM_LAUNCH(P, "k_coefficients", st, k_coefficients<<<nsub, kThreads, 0, st>>>(d.subs, d.faces, K, make_geo(c), c.beta_mode, c.alpha,
                                             c.beta_const, bcm, blo, bhi, coef, scale,
                                             (double*)(ws + L.rhs_part), (double*)(ws + L.face_tr),
                                             (double*)(ws + L.face_beta), t.n_cells));
    if (precision == MRCM_FP64) {
        size_t sm = sizeof(double) * ((size_t)t.max_b * t.max_b + 2 * t.max_b);
        cudaFuncSetAttribute(k_block_factor<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor<double, false><<<nsub, kThreads, sm, st>>>(d.subs, coef, scale, (double*)(ws + L.W),
                                                                 status, t.n_cells, t.max_b));
    } else {
        size_t sm = sizeof(float) * ((size_t)t.max_b * t.max_b + 2 * t.max_b);
        cudaFuncSetAttribute(k_block_factor<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor<float, true><<<nsub, kThreads, sm, st>>>(d.subs, coef, scale, (float*)(ws + L.W),
                                                               status, t.n_cells, t.max_b));
    }
    return (int)cudaGetLastError();
}

int launch_solve_mbf(const Tables& t, const DeviceTables& d, const Layout& L, char* ws,
                     const double* f, int precision, int sweeps, double tol, void* stream, Prof& P) {
    cudaStream_t st = (cudaStream_t)stream;
    const int nsub = (int)t.subs.size();
    Geo geo = make_geo(t.cfg);
    double* X = (double*)(ws + L.X);
    double* R = (double*)(ws + L.R);
    double* coef = (double*)(ws + L.coef);
    double* scale = (double*)(ws + L.scale);
    int* status = (int*)(ws + L.status);
    MRCM_LAUNCH(P, "k_rhs", st, k_rhs<<<nsub, kThreads, 0, st>>>(d.subs, d.faces, (double*)(ws + L.face_tr), (double*)(ws + L.face_beta),
                                    (double*)(ws + L.rhs_part), f, geo, X));
    if (precision == MRCM_FP64) {
        size_t sm = solve_smem<double>(t.max_b, t.max_m);
        cudaFuncSetAttribute(k_block_solve<double, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        MRCM_LAUNCH(P, "k_block_solve", st, k_block_solve<double, false, false><<<nsub, kThreads, sm, st>>>(d.subs, coef, scale,
            (const double*)(ws + L.W), X, X, t.n_cells, nullptr));
        MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_SWEEPS, 0));
    } else {
        size_t sm = solve_smem<float>(t.max_b, t.max_m);
        cudaFuncSetAttribute(k_block_solve<float, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_block_solve<float, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        MRCM_LAUNCH(P, "k_block_solve", st, k_block_solve<float, true, false><<<nsub, kThreads, sm, st>>>(d.subs, coef, scale,
            (const float*)(ws + L.W), X, X, t.n_cells, nullptr));
        for (int it = 0; it < sweeps; ++it) {
            MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_UNCONVERGED, 0));
            MRCM_LAUNCH(P, "k_residual", st, k_residual<<<nsub, kThreads, 0, st>>>(d.subs, d.faces, coef, (double*)(ws + L.face_tr),
                (double*)(ws + L.face_beta), (double*)(ws + L.rhs_part), f, geo, X, R, t.n_cells, tol, status));
            MRCM_LAUNCH(P, "k_block_solve", st, k_block_solve<float, true, true><<<nsub, kThreads, sm, st>>>(d.subs, coef, scale,
                (const float*)(ws + L.W), R, X, t.n_cells, status + ST_UNCONVERGED));
        }
        // final check of the refined columns
        MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_UNCONVERGED, 0));
        MRCM_LAUNCH(P, "k_residual", st, k_residual<<<nsub, kThreads, 0, st>>>(d.subs, d.faces, coef, (double*)(ws + L.face_tr),
            (double*)(ws + L.face_beta), (double*)(ws + L.rhs_part), f, geo, X, R, t.n_cells, tol, status));
        MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_SWEEPS, sweeps));
    }
    MRCM_LAUNCH(P, "k_element", st, k_element<<<nsub, kThreads, 0, st>>>(d.subs, d.faces, (double*)(ws + L.face_tr), (double*)(ws + L.face_beta),
                                        X, geo, (double*)(ws + L.elem), (double*)(ws + L.elem_b)));
    return (int)cudaGetLastError();
}

}  // namespace mrcm
