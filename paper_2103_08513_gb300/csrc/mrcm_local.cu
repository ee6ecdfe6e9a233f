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

#include <algorithm>
#include <cstdint>
#include <type_traits>
#include <vector>

#include "mrcm_devmath.cuh"
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

// Robin coefficient of a face with normal permeability Kn: beta (the constant,
// or alpha H / Kn with H the subdomain's extent along the normal) and
// T_R = A_f / (h_n / (2 Kn) + beta), with one Newton reciprocal of Kn shared by
// both and one of the denominator instead of FP64 divisions.
__device__ __forceinline__ void robin_of(int mode, double alpha, double beta_const, const SubInfo& s, int a,
                                         double h_a, double area_a, double Kn, double* beta, double* tr) {
    const double ik = rcp64(Kn);
    const double be = mode == MRCM_BETA_CONST ? beta_const : alpha * (double)s.sz[a] * h_a * ik;
    *beta = be;
    *tr = area_a * rcp64(fma(0.5 * h_a, ik, be));
}

// ---------------------------------------------------------------------------
// Per-cell coefficients (FP64): diagonal (incl. Robin and Dirichlet terms),
// the three "+" transmissibilities along (u, v, s), the Jacobi scale and the
// Dirichlet part of the particular right-hand side.  Also T_R, beta, the
// U-MBF right-hand side -beta s T_R and beta s T_R of every Robin face.
// Each interior face's transmissibility (area / h) 2 K1 K2 / (K1 + K2) is
// computed once, by the cell on its low side, with a Newton reciprocal (an
// FP64 division is a long chain on this GPU's FP64 unit); the high-side cell
// reads it back after a barrier.  The Jacobi scale 1 / sqrt(diag) only has to
// be a consistent preconditioner, so it is formed in FP32 and widened exactly.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_coefficients(const SubInfo* __restrict__ subs, const FaceInfo* __restrict__ faces,
               const double* __restrict__ K, Geo geo, int beta_mode, double alpha, double beta_const,
               int4 bc_lo_hi /* x: mask of Dirichlet low walls, y: high walls */,
               double3 bc_lo, double3 bc_hi,
               double* __restrict__ coef, double* __restrict__ scale, double* __restrict__ rhs_dir,
               double* __restrict__ face_tr, double* __restrict__ face_beta, double* __restrict__ face_u,
               double* __restrict__ face_bst, long long ncell_total) {
    const SubInfo s = subs[blockIdx.x];
    const long long ncells = (long long)geo.n[0] * geo.n[1] * geo.n[2];
    const double* Kc[3] = {K, K + ncells, K + 2 * ncells};
    const long long stride[3] = {1, geo.n[0], (long long)geo.n[0] * geo.n[1]};
    const double blo[3] = {bc_lo.x, bc_lo.y, bc_lo.z};
    const double bhi[3] = {bc_hi.x, bc_hi.y, bc_hi.z};
    double ah[3];                                      // area / h per axis
    for (int a = 0; a < 3; ++a) ah[a] = geo.area[a] * rcp64(geo.h[a]);
    int lstride[3];                                    // in-subdomain cell stride along each global axis
    lstride[s.ua] = 1; lstride[s.va] = s.su; lstride[s.sa] = s.b;
    double* tp[3];                                     // "+" transmissibility arrays by global axis
    tp[s.ua] = coef + ncell_total + s.cell_off;
    tp[s.va] = coef + 2 * ncell_total + s.cell_off;
    tp[s.sa] = coef + 3 * ncell_total + s.cell_off;
    // pass 1: interior faces, from their low-side cell
    for (int c = threadIdx.x; c < s.N; c += blockDim.x) {
        int lc[3];
        local_coords(s, c, lc);
        const long long g = global_cell(s, lc, geo.n);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double T = 0.0;
            if (lc[a] + 1 < s.sz[a]) {
                const double k1 = Kc[a][g], k2 = Kc[a][g + stride[a]];
                T = 2.0 * ah[a] * k1 * k2 * rcp64(k1 + k2);
            }
            tp[a][c] = T;
        }
    }
    __syncthreads();                                   // the high-side cells read their "-" faces
    for (int c = threadIdx.x; c < s.N; c += blockDim.x) {
        int lc[3];
        local_coords(s, c, lc);
        const long long g = global_cell(s, lc, geo.n);
        double d = 0.0, rd = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // +a side
            if (lc[a] + 1 < s.sz[a]) {
                d += tp[a][c];
            } else if (s.o[a] + lc[a] == geo.n[a] - 1) {
                if ((bc_lo_hi.y >> a) & 1) { double TD = 2.0 * ah[a] * Kc[a][g]; d += TD; rd += TD * bhi[a]; }
            } else {
                double beta, tr;
                robin_of(beta_mode, alpha, beta_const, s, a, geo.h[a], geo.area[a], Kc[a][g], &beta, &tr);
                d += tr;
            }
            // -a side
            if (lc[a] > 0) {
                d += tp[a][c - lstride[a]];
            } else if (s.o[a] == 0) {
                if ((bc_lo_hi.x >> a) & 1) { double TD = 2.0 * ah[a] * Kc[a][g]; d += TD; rd += TD * blo[a]; }
            } else {
                double beta, tr;
                robin_of(beta_mode, alpha, beta_const, s, a, geo.h[a], geo.area[a], Kc[a][g], &beta, &tr);
                d += tr;
            }
        }
        const long long i = s.cell_off + c;
        coef[i] = d;
        scale[i] = f32_to_f64(rsqrtf(f64_to_f32_rz(d)));
        rhs_dir[i] = rd;
    }
    for (int q = threadIdx.x; q < s.nface; q += blockDim.x) {
        FaceInfo fi = faces[s.face_off + q];
        int lc[3];
        local_coords(s, fi.cell, lc);
        long long g = global_cell(s, lc, geo.n);
        int a = fi.axis;
        double beta, tr;
        robin_of(beta_mode, alpha, beta_const, s, a, geo.h[a], geo.area[a], Kc[a][g], &beta, &tr);
        face_tr[s.face_off + q] = tr;
        face_beta[s.face_off + q] = beta;
        face_u[s.face_off + q] = -beta * fi.s * tr;     // U-MBF right-hand side on this face
        face_bst[s.face_off + q] = beta * fi.s * tr;     // weight of the face's flux in the U row
    }
}

// ---------------------------------------------------------------------------
// Slab block factorisation: W_s = S_s^{-1} by in-place Gauss-Jordan on the
// SPD block pivot (no pivoting needed for SPD), one CTA per subdomain.
//
// Gauss-Jordan on a symmetric matrix keeps M[i][j] = sigma_i sigma_j M[j][i]
// with sigma = -1 on the indices already pivoted (the "sweep operator"), so
// only the lower triangle is stored (packed, row i at i(i+1)/2) and updated:
// step k, with r_j = M[k][j] read from the lower triangle and
// c_i = M[i][k] = sigma_i r_i,
//   M[i][j] -= c_i r_j / p  (i, j != k),  M[k][j] = r_j / p,
//   M[i][k] = -c_i / p,  M[k][k] = 1 / p.
// After the last pivot every sigma is -1 and the triangle holds S_s^{-1}.
// W_s is written to global memory as a full b x b matrix.
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t packed_len(int b) { return (size_t)b * (b + 1) / 2; }

template <typename T, bool kScaled>
__global__ void __launch_bounds__(kThreads)
k_block_factor(const SubInfo* __restrict__ subs, const int* __restrict__ list, const double* __restrict__ coef,
               const double* __restrict__ scale, T* __restrict__ Wall, int* __restrict__ status,
               long long nct, float* __restrict__ scf_all, float* __restrict__ tsc_all,
               const int* __restrict__ limit /* CTAs from *limit on have no subdomain; may be NULL */,
               T* __restrict__ big /* packed triangles of the blocks with a global slot; may be NULL */) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (limit && (int)blockIdx.x >= *limit) return;
    const SubInfo s = subs[list[blockIdx.x]];
    const int b = s.b, su = s.su;
    T* rk = reinterpret_cast<T*>(smem_raw);                    // row k
    T* tv = rk + b;                                            // scaled couplings to the previous slab
    // packed lower triangle: shared memory, or the subdomain's global slot (L2-resident) when it is too large
    T* Lp = (big && s.big_slot >= 0) ? big + (size_t)s.big_slot * packed_len(kMaxBlock)
                                     : tv + ((b + 1) & ~1);
    const double* cd = coef + s.cell_off;
    const double* cu = coef + nct + s.cell_off;
    const double* cv = coef + 2 * nct + s.cell_off;
    const double* cs = coef + 3 * nct + s.cell_off;
    const double* sc = scale + s.cell_off;
    T* W = Wall + s.w_off;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;    // 32 x 8 threads
    int bad = 0;
    for (int i = threadIdx.x; i < (int)packed_len(b); i += blockDim.x) Lp[i] = (T)0;
    for (int sl = 0; sl < s.ns; ++sl) {
        const int base = sl * b;
        for (int i = threadIdx.x; i < b; i += blockDim.x) {
            const int c = base + i;
            double t = 0.0;
            if (sl > 0) t = cs[c - b] * (kScaled ? sc[c - b] * sc[c] : 1.0);
            tv[i] = (T)t;
            if (kScaled) {
                scf_all[s.cell_off + c] = (float)sc[c];
                tsc_all[s.cell_off + c] = sl + 1 < s.ns ? (float)(cs[c] * sc[c] * sc[c + b]) : 0.0f;
            }
        }
        __syncthreads();
        // S_s = D_s - t o W_{s-1} o t on the lower triangle
        for (int i = ty; i < b; i += 8) {
            const int ci = base + i;
            const int ui = i % su;
            const double si = kScaled ? sc[ci] : 1.0;
            T* row = Lp + packed_len(i);
            for (int j = tx; j <= i; j += 32) {
                const int cj = base + j;
                double dij = 0.0;
                if (i == j) dij = cd[ci];
                if (i == j + 1 && ui > 0) dij = -cu[cj];
                if (i == j + su) dij = -cv[cj];
                if (kScaled) dij *= si * sc[cj];
                row[j] = (T)(dij - (double)tv[i] * (double)tv[j] * (double)row[j]);
            }
        }
        __syncthreads();
        // sweep operator on the packed triangle
        for (int k = 0; k < b; ++k) {
            for (int j = threadIdx.x; j < b; j += blockDim.x) rk[j] = j <= k ? Lp[packed_len(k) + j] : Lp[packed_len(j) + k];
            __syncthreads();
            T p = rk[k];
            if (!(p > (T)0)) { bad = 1; p = (T)1; }
            const T ip = (T)1 / p;
            for (int i = ty; i < b; i += 8) {
                const T ci = i < k ? -rk[i] : rk[i];
                T* row = Lp + packed_len(i);
                for (int j = tx; j <= i; j += 32) {
                    T v;
                    if (i == k) v = j == k ? ip : rk[j] * ip;
                    else if (j == k) v = -ci * ip;
                    else v = row[j] - ci * rk[j] * ip;
                    row[j] = v;
                }
            }
            __syncthreads();
        }
        // W_s as a full matrix (both triangles)
        T* Ws = W + (long long)sl * wstride<T>(b);
        for (int i = ty; i < b; i += 8) {
            const T* row = Lp + packed_len(i);
            for (int j = tx; j <= i; j += 32) {
                Ws[(long long)i * b + j] = row[j];
                Ws[(long long)j * b + i] = row[j];
            }
        }
        __syncthreads();
    }
    if (bad && threadIdx.x == 0) atomicAdd(&status[ST_NOT_SPD], 1);
}

template <typename T>
size_t factor_smem(int b) { return sizeof(T) * (packed_len(b) + 2 * (size_t)b + 4); }

// ---------------------------------------------------------------------------
// Register-resident variant of the block factorisation for b <= 64 (FP32,
// scaled): a 64-thread CTA per subdomain, thread i holds row i of the running
// block in registers, the pivot row is broadcast through shared memory, and
// W_{s-1} stays in registers for the next block pivot.  Same arithmetic as
// k_block_factor (in-place Gauss-Jordan without pivoting on the SPD block).
// ---------------------------------------------------------------------------
constexpr int kRegMaxB = 64;

__global__ void __launch_bounds__(kRegMaxB)
k_block_factor_reg(const SubInfo* __restrict__ subs, const int* __restrict__ list, const double* __restrict__ coef,
                   const double* __restrict__ scale, float* __restrict__ Wall, int* __restrict__ status,
                   long long nct, float* __restrict__ scf_all, float* __restrict__ tsc_all) {
    const SubInfo s = subs[list[blockIdx.x]];
    const int b = s.b, su = s.su;
    const int i = threadIdx.x;
    const bool live = i < b;
    const double* cd = coef + s.cell_off;
    const double* cu = coef + nct + s.cell_off;
    const double* cv = coef + 2 * nct + s.cell_off;
    const double* cs = coef + 3 * nct + s.cell_off;
    const double* sc = scale + s.cell_off;
    float* W = Wall + s.w_off;
    float* scf = scf_all + s.cell_off;
    float* tsc = tsc_all + s.cell_off;
    __shared__ __align__(16) float prow[kRegMaxB];
    __shared__ float tv[kRegMaxB];
    float a[kRegMaxB];
#pragma unroll
    for (int j = 0; j < kRegMaxB; ++j) a[j] = 0.0f;
    int bad = 0;
    for (int sl = 0; sl < s.ns; ++sl) {
        const int base = sl * b;
        float dd = 0.f, du = 0.f, dul = 0.f, dv = 0.f, dvl = 0.f, ti = 0.f;
        if (live) {
            const int c = base + i;
            const int u = i % su;
            dd = (float)(cd[c] * sc[c] * sc[c]);
            if (u + 1 < su) du = (float)(-cu[c] * sc[c] * sc[c + 1]);
            if (u > 0) dul = (float)(-cu[c - 1] * sc[c] * sc[c - 1]);
            if (i + su < b) dv = (float)(-cv[c] * sc[c] * sc[c + su]);
            if (i >= su) dvl = (float)(-cv[c - su] * sc[c] * sc[c - su]);
            if (sl > 0) ti = (float)(cs[c - b] * sc[c - b] * sc[c]);
            scf[c] = (float)sc[c];
            tsc[c] = sl + 1 < s.ns ? (float)(cs[c] * sc[c] * sc[c + b]) : 0.0f;
        }
        tv[i] = ti;
        __syncthreads();
        // S_s = D_s - t o W_{s-1} o t   (W_{s-1} in registers; zero at the first slab)
#pragma unroll
        for (int j = 0; j < kRegMaxB; ++j) {
            if (j < b) {
                // independent terms: with su == 1 the u- and v-neighbours share an index
                // (the u-coupling is then zero)
                float v = -ti * tv[j] * a[j];
                if (j == i) v += dd;
                if (j == i + 1) v += du;
                if (j == i - 1) v += dul;
                if (j == i + su) v += dv;
                if (j == i - su) v += dvl;
                a[j] = live ? v : 0.0f;
            }
        }
        // Gauss-Jordan inversion; the pivot row goes through shared memory.
        // Gauss-Jordan on a symmetric matrix keeps M[i][k] = sigma_i M[k][i] with
        // sigma_i = -1 for the columns already pivoted (i < k), +1 otherwise, so
        // each thread reads its column-k entry back from the published row.
#pragma unroll 1
        for (int k = 0; k < b; ++k) {
            __syncthreads();                                 // previous step done with prow
            if (i == k) {
                float4* pr4 = reinterpret_cast<float4*>(prow);
#pragma unroll
                for (int j = 0; j < kRegMaxB; j += 4) pr4[j >> 2] = make_float4(a[j], a[j + 1], a[j + 2], a[j + 3]);
            }
            __syncthreads();
            float p = prow[k];
            if (!(p > 0.0f)) { bad = 1; p = 1.0f; }
            const float ip = 1.0f / p;
            const float ck = i < k ? -prow[i] : prow[i];     // M[i][k]
            const bool own = i == k;
            const float4* pr4 = reinterpret_cast<const float4*>(prow);
#pragma unroll
            for (int j4 = 0; j4 < kRegMaxB; j4 += 4) {
                if (j4 < b) {
                    const float4 q = pr4[j4 >> 2];
                    const float pq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int j = j4 + t;
                        const float tj = pq[t] * ip;
                        if (j == k) a[j] = own ? ip : -ck * ip;
                        else a[j] = own ? tj : fmaf(-ck, tj, a[j]);
                    }
                }
            }
        }
        // store W_s (symmetric: thread i writes column i = row i), coalesced over threads
        float* Ws = W + (long long)sl * wstride<float>(b);
        if (live) {
#pragma unroll
            for (int j = 0; j < kRegMaxB; ++j)
                if (j < b) Ws[j * b + i] = a[j];
        }
        __syncthreads();
    }
    if (bad) atomicAdd(&status[ST_NOT_SPD], 1);
}

// ---------------------------------------------------------------------------
// Register-tiled variant for 64 < b <= 128 (FP32, scaled): 256 threads as a
// 16 x 16 grid, thread (ty, tx) holds the 8 x 8 tile of rows 8 ty .. 8 ty + 7
// and columns 8 tx .. 8 tx + 7 of the running block (rows and columns >= b
// stay zero and are never pivoted).  Same sweep-operator Gauss-Jordan as the
// kernels above: at step k the pivot row is published in shared memory
// (double-buffered, one barrier per step) and column k is read back through
// the sign symmetry M[i][k] = sigma_i M[k][i].  Every entry takes the generic
// update M[i][j] -= M[i][k] M[k][j] / p; row k and column k are then set
// exactly (M[k][j] / p, -M[i][k] / p and 1 / p).  W_{s-1} stays in the
// registers to form S_s = D_s - t o W_{s-1} o t for the next slab.
// ---------------------------------------------------------------------------
// ---- bulk-copy staging of the W blocks (TMA unit, completion on an mbarrier)
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

// One thread: expect `bytes` on the barrier and start the copy global -> shared.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");     // earlier generic reads of dst done
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier, giving up after about two seconds
// (then the status word records a timeout and the caller stops using the buffer).
constexpr long long kWaitCycles = 4000000000LL;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

// ---------------------------------------------------------------------------
// Tensor-core variant for 64 < b <= 128 (FP32 accuracy from 3xTF32): the
// running block matrix lives in tensor memory (TMEM, 128 lanes = rows x 128
// columns), one thread per row (128 threads).  Pivots are swept 16 at a time
// with the blocked form of the same sign-symmetric Gauss-Jordan sweep
// (P = the 16 pivots, all unswept):
//   M_ij <- M_ij - M_iP M_PP^{-1} M_Pj,  M_Pj <- M_PP^{-1} M_Pj,
//   M_iP <- -M_iP M_PP^{-1},             M_PP <- M_PP^{-1}.
// With R_j = M_PP^{-1} M_Pj = sigma_j M_PP^{-1} M[j][P]^T (sign symmetry) and
// A_i = -M[i][P] (+ e_p on the row of pivot p), one tcgen05.mma D += A R^T
// (M = N = 128, K = 16) performs the trailing update and the new pivot rows
// at once; the pivot columns are then written back from registers.  Each
// operand is split into three TF32 pieces x1 + x2 + x3 and the product is
// taken as the six terms down to 2^-22 relative (six MMAs per K step): the
// two-piece "3xTF32" product leaves about 2^-21 per product, enough error to
// stall the FP64 refinement on ill-conditioned blocks.  M_PP^{-1} (16 x 16,
// SPD) is swept by one warp.  Operands sit in shared memory in the canonical
// K-major layout without swizzle (8-row x 16-byte core matrices, 128 B apart
// along K, 512 B apart along rows).  W_{s-1} stays in TMEM to form S_s.
// Every wait on the MMA completion is bounded; a timeout sets the status word
// and stops the subdomain.
// ---------------------------------------------------------------------------
constexpr int kTcN = 128;      // TMEM tile edge
constexpr int kTcP = 16;       // pivots per block step (MMA K = 2 x 8)
constexpr int kTcSmem = 6 * 8192;       // operand pieces; with the static part, at most 4 CTAs (all of TMEM) per SM

__device__ __forceinline__ uint32_t tc_off(int r, int k) {    // byte offset of (row, k) in a 128 x 16 operand
    return (uint32_t)((r >> 3) * 512 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {   // shared-memory matrix descriptor
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ void tm_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
__device__ __forceinline__ void tm_st16(uint32_t taddr, const float v[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 :: "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                    "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                    "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                    "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                    "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                    "r"(__float_as_uint(v[15]))
                 : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_sync() {      // block barrier that also orders tcgen05 operations
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
// D (TMEM) += A B^T, TF32 operands from shared-memory descriptors, issued by one thread
__device__ __forceinline__ void tc_mma_acc(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, 1, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 :: "r"(dtmem), "l"(da), "l"(db), "r"(idesc) : "memory");
}

__global__ void __launch_bounds__(kTcN, 4)
k_block_factor_tc(const SubInfo* __restrict__ subs, const int* __restrict__ list, const double* __restrict__ coef,
                  const double* __restrict__ scale, float* __restrict__ Wall, int* __restrict__ status,
                  long long nct, float* __restrict__ scf_all, float* __restrict__ tsc_all) {
    extern __shared__ __align__(1024) unsigned char opd[];         // A1..A3, B1..B3 (128 x 16 each, 8 KB)
    __shared__ __align__(16) float mpp[2][kTcP][kTcP];              // M_PP^{-1}, double-buffered
    __shared__ float sd[kTcN], sup[kTcN], svp[kTcN], st[kTcN];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int stop_s;
    const SubInfo s = subs[list[blockIdx.x]];
    const int b = s.b, su = s.su;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i = tid;                                              // this thread's row = TMEM lane
    const double* cd = coef + s.cell_off;
    const double* cu = coef + nct + s.cell_off;
    const double* cv = coef + 2 * nct + s.cell_off;
    const double* cs = coef + 3 * nct + s.cell_off;
    const double* sc = scale + s.cell_off;
    float* W = Wall + s.w_off;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" :: "r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        stop_s = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);     // this warp's lane quarter, column 0
    // instruction descriptor: D F32, A/B TF32, both K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcN >> 4) << 24);
    uint32_t phase = 0;
    int bad = 0;
    {
        float z[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) z[q] = 0.0f;
        for (int c0 = 0; c0 < kTcN; c0 += 16) tm_st16(trow + c0, z);  // W_{-1} = 0
    }
    for (int sl = 0; sl < s.ns; ++sl) {
        const int base = sl * b;
        for (int r = tid; r < kTcN; r += blockDim.x) {
            float d = 0.f, u = 0.f, v = 0.f, t = 0.f;
            if (r < b) {
                const int c = base + r;
                d = (float)(cd[c] * sc[c] * sc[c]);
                if ((r % su) + 1 < su) u = (float)(-cu[c] * sc[c] * sc[c + 1]);
                if (r + su < b) v = (float)(-cv[c] * sc[c] * sc[c + su]);
                if (sl > 0) t = (float)(cs[c - b] * sc[c - b] * sc[c]);
                scf_all[s.cell_off + c] = (float)sc[c];
                tsc_all[s.cell_off + c] = sl + 1 < s.ns ? (float)(cs[c] * sc[c] * sc[c + b]) : 0.0f;
            }
            sd[r] = d; sup[r] = u; svp[r] = v; st[r] = t;
        }
        __syncthreads();
        // S_s = D_s - t o W_{s-1} o t, this thread's row
        for (int c0 = 0; c0 < kTcN; c0 += 16) {
            float v[16];
            tm_ld16(trow + c0, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = c0 + q;
                float x = -st[i] * st[j] * v[q];
                if (j == i) x += sd[i];
                if (j == i + 1) x += sup[i];
                if (j + 1 == i) x += sup[j];
                if (j == i + su) x += svp[i];
                if (j + su == i) x += svp[j];
                v[q] = (i < b && j < b) ? x : 0.0f;
            }
            tm_st16(trow + c0, v);
        }
        tc_sync();
        // blocked sweep, 16 pivots per step
        for (int k0 = 0, blk = 0; k0 < b; k0 += kTcP, ++blk) {
            const int nbk = min(kTcP, b - k0);
            float m[16];
            tm_ld16(trow + k0, m);                                  // M[i][P]
            const int ip = i - k0;                                  // pivot index of this row, if in P
            float (*minv)[kTcP] = mpp[blk & 1];                     // double-buffered M_PP^{-1}
            if (warp == (k0 >> 5)) {
                // the warp holding rows P sweeps M_PP in registers (lane L0 + r owns row r)
                const int L0 = k0 & 31;
                float a[16];
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    a[c] = (ip >= 0 && ip < nbk && c < nbk) ? m[c] : (c == ip ? 1.0f : 0.0f);
#pragma unroll
                for (int q = 0; q < kTcP; ++q) {
                    float rq[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) rq[c] = __shfl_sync(0xffffffffu, a[c], L0 + q);
                    float p = rq[q];
                    if (!(p > 0.0f)) { bad = 1; p = 1.0f; }
                    const float inv = 1.0f / p;
                    const float cr = a[q];
                    if (ip == q) {
#pragma unroll
                        for (int c = 0; c < 16; ++c) a[c] = c == q ? inv : rq[c] * inv;
                    } else {
#pragma unroll
                        for (int c = 0; c < 16; ++c) a[c] = c == q ? -cr * inv : fmaf(-cr, rq[c] * inv, a[c]);
                    }
                }
                if (ip >= 0 && ip < kTcP) {
#pragma unroll
                    for (int c = 0; c < 16; c += 4)
                        *reinterpret_cast<float4*>(&minv[ip][c]) = make_float4(a[c], a[c + 1], a[c + 2], a[c + 3]);
                }
            }
            __syncthreads();
            // operands: A_i = -M[i][P] (+ e_p on pivot rows), R_i = sigma_i M_PP^{-1} M[i][P]^T
            const float sg = i < k0 ? -1.0f : 1.0f;
            float R[16], cnew[16];
#pragma unroll
            for (int p = 0; p < 16; ++p) { R[p] = 0.0f; cnew[p] = 0.0f; }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float4* row = reinterpret_cast<const float4*>(&minv[q][0]);   // row q of M_PP^{-1}
#pragma unroll
                for (int p4 = 0; p4 < 4; ++p4) {
                    const float4 w4 = row[p4];
                    const float wq[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        R[q] = fmaf(wq[t], m[4 * p4 + t], R[q]);        // (M_PP^{-1} m)[q]
                        cnew[4 * p4 + t] = fmaf(-m[q], wq[t], cnew[4 * p4 + t]);   // (-m M_PP^{-1})[p]
                    }
                }
            }
            // three-piece TF32 split x = x1 + x2 + x3 (x1, x2 TF32; x3 below 2^-22 |x|)
#pragma unroll
            for (int p4 = 0; p4 < 4; ++p4) {
                float a1[4], a2[4], a3[4], b1[4], b2[4], b3[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int p = 4 * p4 + t;
                    const float a = -m[p] + (ip == p ? 1.0f : 0.0f);
                    const float r = sg * R[p];
                    a1[t] = tf32_hi(a); a2[t] = tf32_hi(a - a1[t]); a3[t] = (a - a1[t]) - a2[t];
                    b1[t] = tf32_hi(r); b2[t] = tf32_hi(r - b1[t]); b3[t] = (r - b1[t]) - b2[t];
                }
                const uint32_t o = tc_off(i, 4 * p4);
                *reinterpret_cast<float4*>(opd + 0 * 8192 + o) = make_float4(a1[0], a1[1], a1[2], a1[3]);
                *reinterpret_cast<float4*>(opd + 1 * 8192 + o) = make_float4(a2[0], a2[1], a2[2], a2[3]);
                *reinterpret_cast<float4*>(opd + 2 * 8192 + o) = make_float4(a3[0], a3[1], a3[2], a3[3]);
                *reinterpret_cast<float4*>(opd + 3 * 8192 + o) = make_float4(b1[0], b1[1], b1[2], b1[3]);
                *reinterpret_cast<float4*>(opd + 4 * 8192 + o) = make_float4(b2[0], b2[1], b2[2], b2[3]);
                *reinterpret_cast<float4*>(opd + 5 * 8192 + o) = make_float4(b3[0], b3[1], b3[2], b3[3]);
            }
            if (ip >= 0 && ip < kTcP) {                             // pivot rows: row of M_PP^{-1}
#pragma unroll
                for (int p = 0; p < 16; ++p) cnew[p] = minv[ip][p];
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // operands visible to the tensor core
            tc_sync();
            if (tid == 0) {
                const uint32_t o0 = smem_u32(opd);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint32_t ko = o0 + ks * 256;                  // K step of 8 = two core matrices
                    const uint64_t a1d = tc_desc(ko), a2d = tc_desc(ko + 8192), a3d = tc_desc(ko + 2 * 8192);
                    const uint64_t b1d = tc_desc(ko + 3 * 8192), b2d = tc_desc(ko + 4 * 8192), b3d = tc_desc(ko + 5 * 8192);
                    tc_mma_acc(tmem, a2d, b2d, idesc);                  // D += a2 b2 + a3 b1 + a1 b3
                    tc_mma_acc(tmem, a3d, b1d, idesc);                  //    + a2 b1 + a1 b2 + a1 b1
                    tc_mma_acc(tmem, a1d, b3d, idesc);                  // (smallest terms first)
                    tc_mma_acc(tmem, a2d, b1d, idesc);
                    tc_mma_acc(tmem, a1d, b2d, idesc);
                    tc_mma_acc(tmem, a1d, b1d, idesc);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(smem_u32(&bar)) : "memory");
            }
            const bool tout = !mbar_wait(&bar, phase);             // bounded: about two seconds
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // new pivot columns (the operands are consumed: the MMA has completed)
            tm_st16(trow + k0, cnew);
            // one decision for the whole CTA (a timeout in any thread stops the subdomain)
            if (__syncthreads_or(tout)) {
                if (tid == 0) { atomicAdd(&status[ST_TIMEOUT], 1); stop_s = 1; }
                break;
            }
        }
        tc_sync();
        if (stop_s) break;
        // W_s: row i of the swept matrix (every lane loads: the TMEM loads are warp-collective)
        {
            float* row = W + (long long)sl * wstride<float>(b) + (long long)min(i, b - 1) * b;
            for (int c0 = 0; c0 < kTcN; c0 += 16) {
                float v[16];
                tm_ld16(trow + c0, v);
                if (i < b) {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (c0 + q < b) row[c0 + q] = v[q];
                }
            }
        }
        tc_sync();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (__syncthreads_or(bad) && tid == 0) atomicAdd(&status[ST_NOT_SPD], 1);   // any warp's pivot
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" :: "r"(tmem));
}

// ---------------------------------------------------------------------------
// Register-tiled variant for 128 < b <= 256 (FP32, scaled): the block is held
// as 8 x 8 tiles of its lower triangle, one tile per thread (at most 32 x 33 /
// 2 = 528 tiles; diagonal tiles keep their full 8 x 8 block).  Pivot k needs
// the row M[k][:] of the sign-symmetric matrix: the threads of tile row k/8
// publish M[k][x] for x in or left of the diagonal tile, the threads of tile
// column k/8 publish M[x][k] = M[k][x] (both unswept) for x below it.  Column
// k is read back as M[i][k] = sigma_i M[k][i].  Each thread then applies the
// same sweep-operator step to its tile; W_s is written as a full matrix.
// ---------------------------------------------------------------------------
constexpr int kTriB = 256;                 // largest block

// CTA size of the triangle factor for a b x b block: whole warps covering the
// nt (nt + 1) / 2 tiles; 0 = beyond kTriB (packed kernel)
static int tri_threads(int b) {
    const int nt = (b + 7) / 8, T = nt * (nt + 1) / 2;
    return b > kTriB ? 0 : T <= 192 ? 192 : T <= 320 ? 320 : T <= 512 ? 512 : 544;
}

// NTH threads: 192 cover b <= 144, 320 b <= 192, 512 b <= 248 (496 tiles),
// all within 128 registers; 544 cover b <= 256 (528 tiles) but then have to
// live with 96 registers (5 warps on one SM sub-partition).
template <int NTH>
__global__ void __launch_bounds__(NTH, NTH <= 192 ? 2 : 1)
k_block_factor_tri(const SubInfo* __restrict__ subs, const int* __restrict__ list, const double* __restrict__ coef,
                   const double* __restrict__ scale, float* __restrict__ Wall, int* __restrict__ status,
                   long long nct, float* __restrict__ scf_all, float* __restrict__ tsc_all) {
    const SubInfo s = subs[list[blockIdx.x]];
    const int b = s.b, su = s.su;
    const int nt = (b + 7) >> 3;
    const int T = nt * (nt + 1) / 2;
    const int t = threadIdx.x;
    const bool own = t < T;
    int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    int tj = t - ti * (ti + 1) / 2;
    if (!own) ti = tj = 0;                                 // idle threads shadow tile (0, 0), never publish or store
    const int i0 = ti * 8, j0 = tj * 8;
    const bool diag = ti == tj;
    const double* cd = coef + s.cell_off;
    const double* cu = coef + nct + s.cell_off;
    const double* cv = coef + 2 * nct + s.cell_off;
    const double* cs = coef + 3 * nct + s.cell_off;
    const double* sc = scale + s.cell_off;
    float* W = Wall + s.w_off;
    __shared__ __align__(16) float prow[2][kTriB];
    __shared__ __align__(16) float sd[kTriB], sup[kTriB], svp[kTriB], st[kTriB];
    float a[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) a[r][c] = 0.0f;
    int bad = 0;
    for (int sl = 0; sl < s.ns; ++sl) {
        const int base = sl * b;
        for (int i = t; i < kTriB; i += NTH) {
            float d = 0.f, u = 0.f, v = 0.f, tt = 0.f;
            if (i < b) {
                const int c = base + i;
                d = (float)(cd[c] * sc[c] * sc[c]);
                if ((i % su) + 1 < su) u = (float)(-cu[c] * sc[c] * sc[c + 1]);
                if (i + su < b) v = (float)(-cv[c] * sc[c] * sc[c + su]);
                if (sl > 0) tt = (float)(cs[c - b] * sc[c - b] * sc[c]);
                scf_all[s.cell_off + c] = (float)sc[c];
                tsc_all[s.cell_off + c] = sl + 1 < s.ns ? (float)(cs[c] * sc[c] * sc[c + b]) : 0.0f;
            }
            sd[i] = d; sup[i] = u; svp[i] = v; st[i] = tt;
        }
        __syncthreads();
        // S_s = D_s - t o W_{s-1} o t on the tile
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int i = i0 + r;
            const float tiv = st[min(i, kTriB - 1)];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int j = j0 + c;
                float v = -tiv * st[min(j, kTriB - 1)] * a[r][c];
                if (j == i) v += sd[i];
                if (j == i + 1) v += sup[i];
                if (j + 1 == i) v += sup[j];
                if (j == i + su) v += svp[i];
                if (j + su == i) v += svp[j];
                a[r][c] = (own && i < b && j < b) ? v : (own && i == j) ? 1.0f : 0.0f;
            }
        }
        // The block is padded to 8 nt with identity pivots, which leave the
        // rest untouched.  Pivots k = 8 kt + kr with kr unrolled, so that row kr and column kr
        // of a tile are fixed registers.  Column k rides on the rank-1 update
        // (zeroed, row factor 1 / p: -M[i][k] / p, and 1 / p at (k, k)); row k
        // takes M[k][j] / p directly.
#pragma unroll 1
        for (int kt = 0; kt < nt; ++kt) {
            const bool rowt = own && ti == kt, colt = own && tj == kt;
#pragma unroll
            for (int kr = 0; kr < 8; ++kr) {
                const int k = kt * 8 + kr;
                float* pr = prow[kr & 1];
                if (rowt) {                                     // M[k][x], x in tiles (kt, tj <= kt)
                    reinterpret_cast<float4*>(pr + j0)[0] = make_float4(a[kr][0], a[kr][1], a[kr][2], a[kr][3]);
                    reinterpret_cast<float4*>(pr + j0)[1] = make_float4(a[kr][4], a[kr][5], a[kr][6], a[kr][7]);
                }
                if (colt && ti > kt) {                          // M[x][k] = M[k][x] for x below the diagonal tile
#pragma unroll
                    for (int r = 0; r < 8; ++r) pr[i0 + r] = a[r][kr];
                }
                __syncthreads();
                float p = pr[k];
                if (!(p > 0.0f)) { bad = 1; p = 1.0f; }
                const float ip = 1.0f / p;
                const float4 q0 = reinterpret_cast<const float4*>(pr + j0)[0], q1 = reinterpret_cast<const float4*>(pr + j0)[1];
                float rkv[8] = {q0.x * ip, q0.y * ip, q0.z * ip, q0.w * ip, q1.x * ip, q1.y * ip, q1.z * ip, q1.w * ip};
                if (colt) {
#pragma unroll
                    for (int r = 0; r < 8; ++r) a[r][kr] = 0.0f;
                    rkv[kr] = ip;
                }
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    float ckr = pr[i0 + r];
                    if (i0 + r < k) ckr = -ckr;                   // M[i][k] = sigma_i M[k][i]
                    if (r == kr && rowt) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) a[r][c] = rkv[c];
                    } else {
#pragma unroll
                        for (int c = 0; c < 8; ++c) a[r][c] = fmaf(-ckr, rkv[c], a[r][c]);
                    }
                }
            }
        }
        // W_s as a full matrix: the tile and, below the diagonal, its transpose
        float* Ws = W + (long long)sl * wstride<float>(b);
        if (own) {
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int i = i0 + r;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int j = j0 + c;
                    if (i < b && j < b) {
                        Ws[(long long)i * b + j] = a[r][c];
                        if (!diag) Ws[(long long)j * b + i] = a[r][c];
                    }
                }
            }
        }
        __syncthreads();
    }
    if (bad) atomicAdd(&status[ST_NOT_SPD], 1);
}

template <int TPT, int G>
__global__ void __launch_bounds__(G * G, G == 16 ? 2 : 8)
k_block_factor_tile(const SubInfo* __restrict__ subs, const int* __restrict__ list, const double* __restrict__ coef,
                    const double* __restrict__ scale, float* __restrict__ Wall, int* __restrict__ status,
                    long long nct, float* __restrict__ scf_all, float* __restrict__ tsc_all) {
    // G x G threads, TPT x TPT entries each
    constexpr int B = TPT * G;                              // largest block covered
    constexpr int NV = TPT / 4;                             // float4 per tile row
    const SubInfo s = subs[list[blockIdx.x]];
    const int b = s.b, su = s.su;
    const int tx = threadIdx.x % G, ty = threadIdx.x / G;
    const int i0 = ty * TPT, j0 = tx * TPT;
    const double* cd = coef + s.cell_off;
    const double* cu = coef + nct + s.cell_off;
    const double* cv = coef + 2 * nct + s.cell_off;
    const double* cs = coef + 3 * nct + s.cell_off;
    const double* sc = scale + s.cell_off;
    float* W = Wall + s.w_off;
    __shared__ __align__(16) float prow[2][B];
    __shared__ __align__(16) float sd[B], sup[B], svp[B], st[B];
    float a[TPT][TPT];
#pragma unroll
    for (int r = 0; r < TPT; ++r)
#pragma unroll
        for (int c = 0; c < TPT; ++c) a[r][c] = 0.0f;
    int bad = 0;
    for (int sl = 0; sl < s.ns; ++sl) {
        const int base = sl * b;
        // scaled diagonal, +u and +v couplings inside the slab, coupling to slab sl - 1
        for (int i = threadIdx.x; i < B; i += blockDim.x) {
            float d = 0.f, u = 0.f, v = 0.f, t = 0.f;
            if (i < b) {
                const int c = base + i;
                d = (float)(cd[c] * sc[c] * sc[c]);
                if ((i % su) + 1 < su) u = (float)(-cu[c] * sc[c] * sc[c + 1]);
                if (i + su < b) v = (float)(-cv[c] * sc[c] * sc[c + su]);
                if (sl > 0) t = (float)(cs[c - b] * sc[c - b] * sc[c]);
                scf_all[s.cell_off + c] = (float)sc[c];
                tsc_all[s.cell_off + c] = sl + 1 < s.ns ? (float)(cs[c] * sc[c] * sc[c + b]) : 0.0f;
            }
            sd[i] = d; sup[i] = u; svp[i] = v; st[i] = t;
        }
        __syncthreads();
        // S_s = D_s - t o W_{s-1} o t
#pragma unroll
        for (int r = 0; r < TPT; ++r) {
            const int i = i0 + r;
            const float ti = st[i];
#pragma unroll
            for (int c = 0; c < TPT; ++c) {
                const int j = j0 + c;
                float v = -ti * st[j] * a[r][c];
                if (j == i) v += sd[i];
                if (j == i + 1) v += sup[i];
                if (j + 1 == i) v += sup[j];
                if (j == i + su) v += svp[i];
                if (j + su == i) v += svp[j];
                a[r][c] = (i < b && j < b) ? v : i == j ? 1.0f : 0.0f;
            }
        }
        // Gauss-Jordan sweep over the b pivots, padded to whole tiles with
        // identity pivots; k = TPT kt + kr with kr unrolled, so that row and
        // column kr of the tile are fixed registers.  Column k rides on the
        // rank-1 update (zeroed, row factor 1 / p); row k takes M[k][j] / p.
        const int ntl = (b + TPT - 1) / TPT;
#pragma unroll 1
        for (int kt = 0; kt < ntl; ++kt) {
            const bool rowt = ty == kt, colt = tx == kt;
#pragma unroll
            for (int kr = 0; kr < TPT; ++kr) {
                const int k = kt * TPT + kr;
                float* pr = prow[kr & 1];
                if (rowt) {
#pragma unroll
                    for (int q = 0; q < NV; ++q)
                        reinterpret_cast<float4*>(pr + j0)[q] =
                            make_float4(a[kr][4 * q], a[kr][4 * q + 1], a[kr][4 * q + 2], a[kr][4 * q + 3]);
                }
                __syncthreads();
                float p = pr[k];
                if (!(p > 0.0f)) { bad = 1; p = 1.0f; }
                const float ip = 1.0f / p;
                float rkv[TPT];
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    const float4 qv = reinterpret_cast<const float4*>(pr + j0)[q];
                    rkv[4 * q] = qv.x * ip; rkv[4 * q + 1] = qv.y * ip; rkv[4 * q + 2] = qv.z * ip; rkv[4 * q + 3] = qv.w * ip;
                }
                if (colt) {
#pragma unroll
                    for (int r = 0; r < TPT; ++r) a[r][kr] = 0.0f;
                    rkv[kr] = ip;
                }
#pragma unroll
                for (int r = 0; r < TPT; ++r) {
                    float ckr = pr[i0 + r];
                    if (i0 + r < k) ckr = -ckr;                   // M[i][k] = sigma_i M[k][i]
                    if (r == kr && rowt) {
#pragma unroll
                        for (int c = 0; c < TPT; ++c) a[r][c] = rkv[c];
                    } else {
#pragma unroll
                        for (int c = 0; c < TPT; ++c) a[r][c] = fmaf(-ckr, rkv[c], a[r][c]);
                    }
                }
            }
        }
        // store W_s (full symmetric matrix, row major)
        float* Ws = W + (long long)sl * wstride<float>(b);
#pragma unroll
        for (int r = 0; r < TPT; ++r) {
            const int i = i0 + r;
            if (i < b) {
                float* row = Ws + (long long)i * b + j0;
                if ((b & 3) == 0 && j0 + TPT <= b) {
#pragma unroll
                    for (int q = 0; q < NV; ++q)
                        reinterpret_cast<float4*>(row)[q] = make_float4(a[r][4 * q], a[r][4 * q + 1], a[r][4 * q + 2], a[r][4 * q + 3]);
                } else {
#pragma unroll
                    for (int c = 0; c < TPT; ++c)
                        if (j0 + c < b) row[c] = a[r][c];
                }
            }
        }
        __syncthreads();
    }
    if (bad && threadIdx.x == 0) atomicAdd(&status[ST_NOT_SPD], 1);
}

// ---------------------------------------------------------------------------
// Multi-RHS block solve, fused with the right-hand sides (first solve) or with
// the FP64 residual (refinement sweep).  One CTA per subdomain.
//
//   first solve (kSweep = false):  r = B                     X  = S x
//   refinement  (kSweep = true):   r = B - A X   (FP64)      X += S x
// where x solves A^ x = S r slab by slab:
//   forward   Z_s = S r_s + t_{s-1} o Y_{s-1},  Y_s = W_s Z_s
//   backward  x_s = Y_s + W_s (t_s o x_{s+1})
// (S = I in the unscaled FP64 mode).  B is built on the fly: the particular
// column holds f V plus the Dirichlet wall terms; P-MBF column k holds T_R on
// the faces of basis k and U-MBF column k holds -beta s T_R there.
//
// Only the columns not yet converged take part (compacted list); in a
// refinement sweep each column's ||r||_2 is compared with tol ||b||_2 and the
// column is retired for later sweeps once it passes.  Y_s is kept in a
// workspace array of type T between the two sweeps.
// ---------------------------------------------------------------------------

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_16a; };

template <typename T>
__device__ __forceinline__ typename Vec4<T>::type ld4(const T* p) { return *reinterpret_cast<const typename Vec4<T>::type*>(p); }

// Y[i][jj] = sum_k W[k][i] Z[k][jj] for i < b, jj < na; thread tile RT rows x 4
// columns (rows i0, i0 + bh, ..., bh = ceil(b / RT)).  Results are handed to
// `store(i, jj, value)`.
template <int RT, typename Store>
__device__ __forceinline__ void block_gemm_sh(const float* Wsm, const float* Z, int b, int na, int mpad, Store store);

template <typename T, int RT, typename Store>
__device__ __forceinline__ void block_gemm(const T* __restrict__ Wsm, const T* __restrict__ Z, int b, int na,
                                           int mpad, Store store) {
    if constexpr (std::is_same<T, float>::value && RT <= 2) {   // (four rows per thread would spill)
        if (__isShared(Wsm)) {                    // staged W block (otherwise W is read from global memory)
            block_gemm_sh<RT>(Wsm, Z, b, na, mpad, store);
            return;
        }
    }
    const int bh = (b + RT - 1) / RT;
    const int mq = (na + 3) >> 2;
    for (int task = threadIdx.x; task < bh * mq; task += blockDim.x) {
        const int i0 = task % bh, cq = task / bh;
        T acc[RT][4];
#pragma unroll
        for (int r = 0; r < RT; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = (T)0;
        const T* zc = Z + 4 * cq;
        for (int k = 0; k < b; ++k) {
            const typename Vec4<T>::type z = ld4(zc + k * mpad);
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const int i = i0 + r * bh;
                const T w = i < b ? Wsm[k * b + i] : (T)0;
                acc[r][0] += w * z.x; acc[r][1] += w * z.y; acc[r][2] += w * z.z; acc[r][3] += w * z.w;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int jj = 4 * cq + q;
            if (jj < na) {
#pragma unroll
                for (int r = 0; r < RT; ++r) {
                    const int i = i0 + r * bh;
                    if (i < b) store(i, jj, acc[r][q]);
                }
            }
        }
    }
}

// block_gemm with both operands in shared memory (FP32): 32-bit shared
// addresses stepped by the row strides.  Rows past the block read row b - 1
// (their sums are never stored), so the loads need no guard.  The same FMAs in
// the same order as the generic form.
template <int RT, typename Store>
__device__ __forceinline__ void block_gemm_sh(const float* Wsm, const float* Z, int b, int na, int mpad, Store store) {
    const int bh = (b + RT - 1) / RT;
    const int mq = (na + 3) >> 2;
    const uint32_t zbase = smem_u32(Z), wbase = smem_u32(Wsm);
    const uint32_t zstep = 4u * (uint32_t)mpad, wstep = 4u * (uint32_t)b;
    for (int task = threadIdx.x; task < bh * mq; task += blockDim.x) {
        const int i0 = task % bh, cq = task / bh;
        float acc[RT][4];
        uint32_t wr[RT];
#pragma unroll
        for (int r = 0; r < RT; ++r) {
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
            wr[r] = wbase + 4u * (uint32_t)min(i0 + r * bh, b - 1);
        }
        uint32_t za = zbase + 16u * (uint32_t)cq, ko = 0;
        for (int k = 0; k < b; ++k) {
            float4 z;
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(z.x), "=f"(z.y), "=f"(z.z), "=f"(z.w) : "r"(za));
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                float w;
                asm volatile("ld.shared.f32 %0, [%1];" : "=f"(w) : "r"(wr[r] + ko));
                acc[r][0] += w * z.x; acc[r][1] += w * z.y; acc[r][2] += w * z.z; acc[r][3] += w * z.w;
            }
            za += zstep;
            ko += wstep;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int jj = 4 * cq + q;
            if (jj < na) {
#pragma unroll
                for (int r = 0; r < RT; ++r) {
                    const int i = i0 + r * bh;
                    if (i < b) store(i, jj, acc[r][q]);
                }
            }
        }
    }
}

// Pair tile (b even): thread tile of rows (i0, i0 + 1) x 4 columns, one
// 2-element load of W and one 4-element load of Z per k for 8 FMAs, no row
// guard (every row pair lies inside the block).
template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// The pair tile with both operands in shared memory (FP32): 32-bit shared
// addresses stepped by the row strides, vector shared loads.  The same FMAs
// in the same order as the generic form below.
template <typename Store>
__device__ __forceinline__ void block_gemm_pair_sh(const float* Wsm, const float* Z, int b, int na, int mpad,
                                                   Store store) {
    const int bh = b >> 1;
    const int mq = (na + 3) >> 2;
    const uint32_t zbase = smem_u32(Z), wbase = smem_u32(Wsm);
    const uint32_t zstep = 4u * (uint32_t)mpad, wstep = 4u * (uint32_t)b;
    for (int task = threadIdx.x; task < bh * mq; task += blockDim.x) {
        const int i0 = 2 * (task % bh), cq = task / bh;
        float a0[4] = {0.f, 0.f, 0.f, 0.f}, a1[4] = {0.f, 0.f, 0.f, 0.f};
        uint32_t za = zbase + 16u * (uint32_t)cq, wa = wbase + 4u * (uint32_t)i0;
#pragma unroll 2
        for (int k = 0; k < b; ++k) {
            float4 z;
            float2 w;
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(z.x), "=f"(z.y), "=f"(z.z), "=f"(z.w) : "r"(za));
            asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(w.x), "=f"(w.y) : "r"(wa));
            za += zstep;
            wa += wstep;
            a0[0] += w.x * z.x; a0[1] += w.x * z.y; a0[2] += w.x * z.z; a0[3] += w.x * z.w;
            a1[0] += w.y * z.x; a1[1] += w.y * z.y; a1[2] += w.y * z.z; a1[3] += w.y * z.w;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int jj = 4 * cq + q;
            if (jj < na) {
                store(i0, jj, a0[q]);
                store(i0 + 1, jj, a1[q]);
            }
        }
    }
}

template <typename T, typename Store>
__device__ __forceinline__ void block_gemm_pair(const T* __restrict__ Wsm, const T* __restrict__ Z, int b, int na,
                                                int mpad, Store store) {
    if constexpr (std::is_same<T, float>::value) {
        if (__isShared(Wsm)) {                    // staged W block (otherwise W is read from global memory)
            block_gemm_pair_sh(Wsm, Z, b, na, mpad, store);
            return;
        }
    }
    const int bh = b >> 1;
    const int mq = (na + 3) >> 2;
    for (int task = threadIdx.x; task < bh * mq; task += blockDim.x) {
        const int i0 = 2 * (task % bh), cq = task / bh;
        T a0[4], a1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { a0[q] = (T)0; a1[q] = (T)0; }
        const T* zc = Z + 4 * cq;
        const T* wc = Wsm + i0;
#pragma unroll 2
        for (int k = 0; k < b; ++k) {
            const typename Vec4<T>::type z = ld4(zc + k * mpad);
            const typename Vec2<T>::type w = *reinterpret_cast<const typename Vec2<T>::type*>(wc + k * b);
            a0[0] += w.x * z.x; a0[1] += w.x * z.y; a0[2] += w.x * z.z; a0[3] += w.x * z.w;
            a1[0] += w.y * z.x; a1[1] += w.y * z.y; a1[2] += w.y * z.z; a1[3] += w.y * z.w;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int jj = 4 * cq + q;
            if (jj < na) {
                store(i0, jj, a0[q]);
                store(i0 + 1, jj, a1[q]);
            }
        }
    }
}

// Tensor-core variant of block_gemm (FP32 operands): warp-level
// mma.sync.m16n8k8 with TF32 inputs and FP32 accumulation, each operand split
// into a TF32 high part and a TF32 remainder, x*y ~ xh*yh + xh*yl + xl*yh
// ("3xTF32"), which keeps FP32-level accuracy on the tensor pipe.  Warps take
// (16-row, 8-column) output tiles; rows >= b and K-padding columns are zero.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float d[4], const uint32_t a[4], const uint32_t bb[2]) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(bb[0]), "r"(bb[1]));
}

template <typename Store>
__device__ __forceinline__ void block_gemm_tc(const float* __restrict__ Wsm, const float* __restrict__ Z, int b,
                                              int na, int mpad, Store store) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    const int mt = (b + 15) >> 4, nt = (na + 7) >> 3, kt = (b + 7) >> 3;
    for (int task = warp; task < mt * nt; task += nwarps) {
        const int m0 = (task % mt) * 16, n0 = (task / mt) * 8;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k8 = 0; k8 < kt; ++k8) {
            const int k0 = k8 * 8;
            float av[4], bv[2];
            const int ar[4] = {m0 + g, m0 + g + 8, m0 + g, m0 + g + 8};
            const int ac[4] = {k0 + tg, k0 + tg, k0 + tg + 4, k0 + tg + 4};
#pragma unroll
            for (int q = 0; q < 4; ++q) av[q] = (ar[q] < b && ac[q] < b) ? Wsm[ac[q] * b + ar[q]] : 0.0f;
            const int br[2] = {k0 + tg, k0 + tg + 4};
            const int bc = n0 + g;
#pragma unroll
            for (int q = 0; q < 2; ++q) bv[q] = (br[q] < b && bc < na) ? Z[br[q] * mpad + bc] : 0.0f;
            uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
            for (int q = 0; q < 4; ++q) { ah[q] = tf32_rna(av[q]); al[q] = tf32_rna(av[q] - __uint_as_float(ah[q])); }
#pragma unroll
            for (int q = 0; q < 2; ++q) { bh[q] = tf32_rna(bv[q]); bl[q] = tf32_rna(bv[q] - __uint_as_float(bh[q])); }
            mma_tf32(acc, al, bh);
            mma_tf32(acc, ah, bl);
            mma_tf32(acc, ah, bh);
        }
        const int r0 = m0 + g, c0 = n0 + 2 * tg;
        if (r0 < b) {
            if (c0 < na) store(r0, c0, acc[0]);
            if (c0 + 1 < na) store(r0, c0 + 1, acc[1]);
        }
        if (r0 + 8 < b) {
            if (c0 < na) store(r0 + 8, c0, acc[2]);
            if (c0 + 1 < na) store(r0 + 8, c0 + 1, acc[3]);
        }
    }
}

// Dispatch: RT > 0 selects the SIMT tile with RT rows per thread, RT == 0 the
// 3xTF32 tensor-core path (FP32 operands only), RT < 0 the pair tile (odd b:
// the one-row tile).
template <typename T, int RT, typename Store>
__device__ __forceinline__ void block_product(const T* Wsm, const T* Z, int b, int na, int mpad, Store store) {
    if constexpr (RT < 0) {
        if (b & 1) block_gemm<T, 1>(Wsm, Z, b, na, mpad, store);
        else block_gemm_pair<T>(Wsm, Z, b, na, mpad, store);
    } else if constexpr (RT == 0) {
        if constexpr (std::is_same<T, float>::value) block_gemm_tc(Wsm, Z, b, na, mpad, store);
    } else {
        block_gemm<T, RT>(Wsm, Z, b, na, mpad, store);
    }
}

// Neighbour flags of a slab cell in the local solve's per-cell mask (bits 0-15: bases mod 16).
constexpr unsigned kNbUp = 1u << 16, kNbUm = 1u << 17, kNbVp = 1u << 18, kNbVm = 1u << 19;

struct LocalArgs {
    const SubInfo* subs;
    const FaceInfo* faces;
    const double* coef;
    const double* scale;
    const float* scf;      // FP32 Jacobi scale (mixed mode)
    const float* tsc;      // FP32 scaled slab coupling (mixed mode)
    const double* face_tr;
    const double* face_beta;
    const double* face_u;
    const double* rhs_dir;
    const double* f;
    Geo geo;
    long long nct;
    double* X;            // MBF array [m][N] per subdomain (FP64)
    void* Ybuf;           // forward-sweep results, type T, same layout as X
    int* conv;            // per column: 1 = converged (skip)
    double* bnorm;        // per column ||b||^2
    double tol2;
    int* status;
    int mpad;             // row stride of the shared column blocks (multiple of 4)
    const int* list;      // subdomains in processing order (costliest first)
    int nlist;
    int* queue;           // work-queue counter (reset to 0 before each launch)
    int count_unconverged;  // add this sweep's unconverged columns to the status word
    int bar_off;          // shared-memory offset of the two mbarriers (after the largest layout)
    int last_only;        // solve only the last (particular) column of every subdomain
    const int* nlist_dev; // when set: the list holds min(nlist, *nlist_dev) subdomains (written by an earlier kernel)
    int col_groups;       // > 1: up to this many CTAs share a subdomain, each taking the columns j = grp mod G
                          // (G = min(col_groups, grid / subdomains)); 1: one CTA per subdomain
    int passes;           // refinement sweeps run back to back on each subdomain by one launch (sweeps only)
};


// Coupling between slab cells c and c+b in the solve's arithmetic: the FP32
// scaled value t^ in mixed mode, the FP64 transmissibility otherwise.
template <typename T, bool kScaled> struct Coupling;
template <> struct Coupling<float, true> {
    const float* tsc; const float* scf;
    __device__ float t(int c) const { return tsc[c]; }
    __device__ float in(double r, int c) const { return f64_to_f32_rz(r) * scf[c]; }
    __device__ float in(double, float rf, int c) const { return rf * scf[c]; }
    __device__ double out(float x, int c) const { return f32_to_f64(x * scf[c]); }
};
template <> struct Coupling<double, false> {
    const double* cs;
    __device__ double t(int c) const { return cs[c]; }
    __device__ double in(double r, int) const { return r; }
    __device__ double in(double r, float, int) const { return r; }
    __device__ double out(double x, int) const { return x; }
};

// Per-CTA state of the W staging pipeline, kept across subdomains (the same
// in every thread).
struct WPipe {
    uint32_t phase[2];     // parity of the next completion of each buffer
    int pending[2];        // a copy into the buffer has been issued and not waited for
    int abort;             // a wait timed out: stop staging
};

template <typename T, bool kScaled, bool kSweep, int NT, int RT>
__device__ __forceinline__ void solve_one(const LocalArgs& g, const T* __restrict__ Wall, int l, int grp, int G,
                                          bool count_unconverged, unsigned char* smem_raw, WPipe& pipe) {
    constexpr int NY = NT / 32;
    const SubInfo s = g.subs[l];
    const int b = s.b, m = s.m, N = s.N, su = s.su, nI = s.nI, mpad = g.mpad;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x NY threads
    const SolveSmem lay = solve_smem_layout<T>(b, mpad, N);
    const int nbuf = lay.nbuf;                                 // W buffers (0: read W from global memory)
    const long long wsd = wstride<T>(b);
    const size_t wbytes = sizeof(T) * (size_t)wsd;
    T* Wb[2] = {reinterpret_cast<T*>(smem_raw + lay.w), reinterpret_cast<T*>(smem_raw + lay.w + ((wbytes + 127) & ~size_t(127)))};
    T* Z = reinterpret_cast<T*>(smem_raw + lay.z);             // b x mpad, cell-major
    T* Yp = reinterpret_cast<T*>(smem_raw + lay.yp);           // b x mpad: Y_{s-1} / x_{s+1}
    // per active column: squared norm (FP32) of b (first solve) or of r / ||b|| (sweep), and 1 / ||b||
    float* nrm = reinterpret_cast<float*>(smem_raw + lay.nrm);
    float* rsb = nrm + mpad;
    int* cols = reinterpret_cast<int*>(smem_raw + lay.cols);   // active columns
    short* cf = reinterpret_cast<short*>(smem_raw + lay.cf);   // Robin face per (cell, axis, side), -1 = none
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + g.bar_off);
    __shared__ int na_s, abort_s;

    const double* cd = g.coef + s.cell_off;
    const double* cu = g.coef + g.nct + s.cell_off;
    const double* cv = g.coef + 2 * g.nct + s.cell_off;
    const double* cs = g.coef + 3 * g.nct + s.cell_off;
    Coupling<T, kScaled> cp;
    if constexpr (kScaled) { cp.tsc = g.tsc + s.cell_off; cp.scf = g.scf + s.cell_off; }
    else { cp.cs = cs; }
    const T* W = Wall + s.w_off;
    double* Xs = g.X + s.x_off;
    T* Ys = reinterpret_cast<T*>(g.Ybuf) + s.y_off;
    int* conv = g.conv + s.rhs_off;
    const double vol = g.geo.h[0] * g.geo.h[1] * g.geo.h[2];

    // active columns (deterministic compaction by one warp)
    if (threadIdx.x < 32) {
        int base = 0;
        for (int j0 = 0; j0 < m; j0 += 32) {
            const int j = j0 + threadIdx.x;
            const bool act = j < m && (!g.last_only || j == m - 1) && (!kSweep || conv[j] == 0) &&
                             (G == 1 || j % G == grp);
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            if (act) cols[base + __popc(bal & ((1u << threadIdx.x) - 1u))] = j;
            base += __popc(bal);
        }
        if (threadIdx.x == 0) na_s = base;
    }
    __syncthreads();
    const int na = na_s;
    if (na == 0) { __syncthreads(); return; }      // nothing left to refine here (before any set-up work)
    for (int e = threadIdx.x; e < 6 * N; e += blockDim.x) cf[e] = -1;
    for (int e = threadIdx.x; e < mpad; e += blockDim.x) {
        nrm[e] = 0.0f;
        float sc = 1.0f;
        if (kSweep && e < na) {
            const float bn = (float)g.bnorm[s.rhs_off + cols[e]];
            if (bn > 0.0f) sc = rsqrtf(bn);
        }
        rsb[e] = sc;
    }
    __syncthreads();                               // cf cleared before the faces are entered
    for (int q = threadIdx.x; q < s.nface; q += blockDim.x) {
        const FaceInfo fi = g.faces[s.face_off + q];
        cf[6 * fi.cell + 2 * fi.axis + (fi.s > 0 ? 1 : 0)] = (short)q;   // one face per cell side
    }
    // W block sequence: forward W_0 .. W_{ns-1}, backward W_{ns-2} .. W_0
    const int nq = 2 * s.ns - 1;
    auto blk = [&](int q) { return q < s.ns ? q : 2 * s.ns - 2 - q; };
    const bool staged = nbuf > 0 && !pipe.abort;
    if (threadIdx.x == 0) abort_s = 0;
    if (staged) {
        for (int q = 0; q < nbuf && q < nq; ++q) {
            if (threadIdx.x == 0) bulk_load(Wb[q], W + blk(q) * wsd, (uint32_t)wbytes, &bar[q]);
            pipe.pending[q] = 1;
        }
    }
    __syncthreads();
    // The block of step q (staged: wait for its copy), and the refill after use.
    auto wblock = [&](int q) -> const T* {
        if (!staged) return W + blk(q) * wsd;
        const int bi = q % nbuf;
        if (pipe.pending[bi]) {
            if (mbar_wait(&bar[bi], pipe.phase[bi])) {
                pipe.phase[bi] ^= 1u;
                pipe.pending[bi] = 0;
            } else {
                if (threadIdx.x == 0) atomicAdd(&g.status[ST_TIMEOUT], 1);
                abort_s = 1;
            }
        }
        return Wb[bi];
    };
    auto refill = [&](int q) {                     // after the block of step q has been used (post-barrier)
        const int bi = q % nbuf;
        if (staged && q + nbuf < nq && !abort_s && !pipe.pending[bi]) {
            if (threadIdx.x == 0) bulk_load(Wb[bi], W + blk(q + nbuf) * wsd, (uint32_t)wbytes, &bar[bi]);
            pipe.pending[bi] = 1;
        }
    };

    // one slab's stencil coefficients, staged per slab for the refinement residual:
    // diagonal, +u, +v, +slab and -slab transmissibilities
    double* co_d = reinterpret_cast<double*>(smem_raw + lay.co);
    double* co_u = co_d + b;
    double* co_v = co_u + b;
    double* co_sp = co_v + b;
    double* co_sm = co_sp + b;
    // the slab's Jacobi scale (mixed mode) and its coupling to the neighbouring slab of the sweep
    T* t_s = reinterpret_cast<T*>(co_sm + b);
    float* sc_s = reinterpret_cast<float*>(t_s + b);
    // per slab cell: bits 0-15 flag the bases (mod 16) of its Robin faces, bits 16-19 which
    // in-slab neighbours exist (+u, -u, +v, -v)
    unsigned* msk_s = reinterpret_cast<unsigned*>(sc_s + b);
    signed char* fcol_s = reinterpret_cast<signed char*>(msk_s + b);  // basis column of each cell side's face, -1 none
    auto stage_slab = [&](int base, int nb_off) {       // nb_off: -b (forward), +b (backward)
        for (int i = threadIdx.x; i < b; i += blockDim.x) {
            const int c = base + i;
            if constexpr (kScaled) sc_s[i] = cp.scf[c];
            const int ct = nb_off < 0 ? c - b : c;
            t_s[i] = (nb_off < 0 ? c >= b : c + b < N) ? cp.t(ct) : (T)0;
            if (nb_off < 0) {
                const int u = i % su;
                unsigned mk = (u + 1 < su ? kNbUp : 0u) | (u > 0 ? kNbUm : 0u) | (i + su < b ? kNbVp : 0u) |
                              (i >= su ? kNbVm : 0u);
#pragma unroll
                for (int a = 0; a < 6; ++a) {
                    const int q = cf[6 * c + a];
                    const int col = q >= 0 ? g.faces[s.face_off + q].col : -1;
                    fcol_s[6 * i + a] = (signed char)col;
                    if (col >= 0) mk |= 1u << (col & 15);
                }
                msk_s[i] = mk;
            }
        }
    };
    auto zin = [&](double r, float rf, int i) -> T {
        if constexpr (kScaled) return rf * sc_s[i];
        else return (T)r;
    };
    auto xout = [&](T x, int i) -> double {
        if constexpr (kScaled) return f32_to_f64(x * sc_s[i]);
        else return (double)x;
    };
    // ---- forward sweep
    for (int sl = 0; sl < s.ns; ++sl) {
        const int base = sl * b;
        if constexpr (kSweep) {
            for (int i = threadIdx.x; i < b; i += blockDim.x) {
                const int c = base + i;
                co_d[i] = cd[c];
                co_u[i] = cu[c];
                co_v[i] = cv[c];
                co_sp[i] = c + b < N ? cs[c] : 0.0;
                co_sm[i] = c >= b ? cs[c - b] : 0.0;
            }
        }
        stage_slab(base, -b);
        __syncthreads();
        // r = B (- A X) of the slab in FP64, its squared norm, and Z = S r + t^ o Y_{s-1}.
        // The (cell i, active column jj) entries are spread over the whole CTA, column by
        // column (a warp reads consecutive cells); each entry's squared norm is parked in
        // Yp[i][jj] by the thread that has just read Y_{s-1} there, and the columns' sums
        // are taken afterwards in a fixed order.
        {
            int jj = threadIdx.x / b, i = threadIdx.x - jj * b;
            const int dj = NT / b, di = NT - dj * b;
            for (int e = threadIdx.x; e < na * b; e += NT) {
                const int j = cols[jj];
                const int c = base + i;
                const unsigned mk = msk_s[i];
                double r;
                if (j == m - 1) {
                    int lc[3];
                    local_coords(s, c, lc);
                    r = g.rhs_dir[s.cell_off + c] + g.f[global_cell(s, lc, g.geo.n)] * vol;
                } else {
                    // MBF column of basis kb (P for j < nI, U after): the value on the one Robin
                    // face of this cell that carries kb, if any (faces of one cell belong to
                    // different bases); the mask rules out most cells, moves only
                    r = 0.0;
                    const int kb = j < nI ? j : j - nI;
                    if ((mk >> (kb & 15)) & 1u) {
#pragma unroll
                        for (int a = 0; a < 6; ++a)
                            if (fcol_s[6 * i + a] == kb) {
                                const int q = s.face_off + cf[6 * c + a];
                                r = j < nI ? g.face_tr[q] : g.face_u[q];
                            }
                    }
                }
                if (kSweep) {                     // r - A x as one FMA chain
                    const double* x = Xs + (long long)j * N;
                    r = fma(-co_d[i], x[c], r);
                    if (mk & kNbUp) r = fma(co_u[i], x[c + 1], r);
                    if (mk & kNbUm) r = fma(co_u[i - 1], x[c - 1], r);
                    if (mk & kNbVp) r = fma(co_v[i], x[c + su], r);
                    if (mk & kNbVm) r = fma(co_v[i - su], x[c - su], r);
                    if (c + b < N) r = fma(co_sp[i], x[c + b], r);
                    if (c >= b) r = fma(co_sm[i], x[c - b], r);
                }
                const float rf = f64_to_f32_rz(r);
                const float rn = rf * rsb[jj];
                T z = zin(r, rf, i);
                T* yp = &Yp[i * mpad + jj];
                if (sl > 0) z += t_s[i] * *yp;
                Z[i * mpad + jj] = z;
                *yp = (T)(rn * rn);
                i += di;
                jj += dj;
                if (i >= b) { i -= b; ++jj; }
            }
        }
        __syncthreads();
        for (int jj = ty; jj < na; jj += NY) {
            float rr = 0.0f;
            for (int i = tx; i < b; i += 32) rr += (float)Yp[i * mpad + jj];
            for (int o = 16; o > 0; o >>= 1) rr += __shfl_down_sync(0xffffffffu, rr, o);
            if (tx == 0) nrm[jj] += rr;          // fixed order per column
        }
        const T* Wsm = wblock(sl);
        __syncthreads();
        block_product<T, RT>(Wsm, Z, b, na, mpad, [&](int i, int jj, T v) {
            Yp[i * mpad + jj] = v;
            Ys[(g.last_only ? 0 : (long long)cols[jj] * N) + base + i] = v;
        });
        __syncthreads();
        refill(sl);
    }
    // ---- backward sweep (Yp holds x_{s+1})
    for (int sl = s.ns - 1; sl >= 0; --sl) {
        const int base = sl * b;
        const bool last = sl == s.ns - 1;
        stage_slab(base, b);
        __syncthreads();
        auto finish = [&](int i, int jj, T acc) {
            const int j = cols[jj];
            const long long gi = (long long)j * N + base + i;
            const T x = Ys[(g.last_only ? 0 : (long long)j * N) + base + i] + acc;
            Yp[i * mpad + jj] = x;                 // Z, not Yp, feeds the product
            const double xo = xout(x, i);
            if (kSweep) Xs[gi] += xo; else Xs[gi] = xo;
        };
        if (!last) {
            const int q = 2 * s.ns - 2 - sl;
            for (int e = threadIdx.x; e < na * b; e += NT) {
                const int jj = e / b, i = e - jj * b;
                Z[i * mpad + jj] = t_s[i] * Yp[i * mpad + jj];
            }
            const T* Wsm = wblock(q);
            __syncthreads();
            block_product<T, RT>(Wsm, Z, b, na, mpad, finish);
            __syncthreads();
            refill(q);
        } else {
            for (int e = threadIdx.x; e < na * b; e += NT) {
                const int jj = e / b, i = e - jj * b;
                finish(i, jj, (T)0);
            }
            __syncthreads();
        }
    }
    // convergence bookkeeping
    if (kSweep) {
        __shared__ int nbad;
        if (threadIdx.x == 0) {
            nbad = 0;
            atomicAdd(reinterpret_cast<unsigned long long*>(g.status + ST_SWEPT), (unsigned long long)na * N);
        }
        __syncthreads();
        for (int jj = threadIdx.x; jj < na; jj += blockDim.x) {
            const int j = cols[jj];
            if (nrm[jj] <= (float)g.tol2) conv[j] = 1;          // ||r||^2 / ||b||^2 <= tol^2
            else atomicAdd(&nbad, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0 && nbad && count_unconverged) atomicAdd(&g.status[ST_UNCONVERGED], nbad);
    } else {
        for (int jj = threadIdx.x; jj < na; jj += blockDim.x) {
            const int j = cols[jj];
            g.bnorm[s.rhs_off + j] = (double)nrm[jj];
            conv[j] = 0;
        }
    }
    __syncthreads();                              // shared memory is reused by the next subdomain
    pipe.abort = abort_s;
}

// Before a CTA leaves: wait (bounded) for copies still in flight into its
// buffers, which only a timed-out wait can leave behind.
__device__ __forceinline__ void drain_pipe(WPipe& pipe, unsigned long long* bar) {
    for (int bi = 0; bi < 2; ++bi)
        if (pipe.pending[bi]) mbar_wait(&bar[bi], pipe.phase[bi]);
}

// Persistent local solve: CTAs pull subdomains from a device work queue over
// the cost-ordered list until it is exhausted (no waits: a plain atomic counter).
template <typename T, bool kScaled, bool kSweep, int NT, int RT>
__global__ void __launch_bounds__(NT, 1280 / NT)       // <= 51 (64 at 512 threads) registers per thread
k_local_solve(LocalArgs g, const T* __restrict__ Wall) {
    extern __shared__ __align__(128) unsigned char smem_ls[];
    unsigned char* smem_raw = smem_ls;
    __shared__ int item;
    // mbarriers at the end of the largest layout (every subdomain's layout places them below)
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + g.bar_off);
    if (threadIdx.x == 0) { mbar_init(&bar[0]); mbar_init(&bar[1]); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    WPipe pipe;
    pipe.phase[0] = pipe.phase[1] = 0u;
    pipe.pending[0] = pipe.pending[1] = 0;
    pipe.abort = 0;
    const int nlist = g.nlist_dev ? min(g.nlist, *g.nlist_dev) : g.nlist;
    const int G = g.col_groups <= 1 || nlist <= 0 ? 1 : max(1, min(g.col_groups, (int)gridDim.x / nlist));
    for (;;) {
        if (threadIdx.x == 0) item = atomicAdd(g.queue, 1);
        __syncthreads();
        const int it = item;
        __syncthreads();
        if (it >= nlist * G || pipe.abort) break;
        // sweeps: g.passes passes on this subdomain back to back (the columns retired by one
        // pass, written to conv[] before the pass's last barrier, drop out of the next)
        const int np = kSweep ? max(1, g.passes) : 1;
        for (int ps = 0; ps < np && !pipe.abort; ++ps)
            solve_one<T, kScaled, kSweep, NT, RT>(g, Wall, g.list[it / G], it % G, G,
                                                  g.count_unconverged && ps + 1 == np, smem_raw, pipe);
    }
    drain_pipe(pipe, bar);
}

// Tunable variants of the local solve: threads per CTA x block-product path
// (SIMT with 2, 1 or 4 rows per thread, the pair tile, or 3xTF32 tensor
// cores for FP32).
constexpr int kNumSolveVariants = 12;
static_assert(kNumSolveVariants <= kMaxSolveVariants, "per-variant tables are too small");
__host__ __device__ inline int variant_threads(int v) {
    return v == 10 ? 256 : v == 11 ? 128 : v >= 8 ? 512 : v == 6 ? 256 : v == 7 ? 128 : v < 3 ? 256 : 128;
}

template <typename T, bool kScaled, bool kSweep>
const void* solve_kernel(int v) {
    switch (v) {
        case 0: return (const void*)k_local_solve<T, kScaled, kSweep, 256, 2>;
        case 1: return (const void*)k_local_solve<T, kScaled, kSweep, 256, 1>;
        case 2: return (const void*)k_local_solve<T, kScaled, kSweep, 256, 4>;
        case 3: return (const void*)k_local_solve<T, kScaled, kSweep, 128, 2>;
        case 4: return (const void*)k_local_solve<T, kScaled, kSweep, 128, 1>;
        case 5: return (const void*)k_local_solve<T, kScaled, kSweep, 128, 4>;
        case 6:
            if constexpr (std::is_same<T, float>::value) return (const void*)k_local_solve<T, kScaled, kSweep, 256, 0>;
            else return (const void*)k_local_solve<T, kScaled, kSweep, 256, 2>;
        case 7:
            if constexpr (std::is_same<T, float>::value) return (const void*)k_local_solve<T, kScaled, kSweep, 128, 0>;
            else return (const void*)k_local_solve<T, kScaled, kSweep, 128, 2>;
        case 8: return (const void*)k_local_solve<T, kScaled, kSweep, 512, 2>;
        case 10: return (const void*)k_local_solve<T, kScaled, kSweep, 256, -2>;
        case 11: return (const void*)k_local_solve<T, kScaled, kSweep, 128, -2>;
        default: return (const void*)k_local_solve<T, kScaled, kSweep, 512, 1>;
    }
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
          const double* __restrict__ face_bst, const double* __restrict__ X, Geo geo,
          double* __restrict__ elem, double* __restrict__ elem_b, int jb_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SubInfo s = subs[blockIdx.x];
    const int nI = s.nI, m = s.m, N = s.N, dim = s.el_dim, nf = s.nface;
    // the subdomain's face cells and weights, staged once; then the face
    // cells' values of jb_max MBF columns at a time
    double* s_tr = reinterpret_cast<double*>(smem_raw);
    double* s_bst = s_tr + nf;
    double* s_be = s_bst + nf;
    double* xs = s_be + nf;                           // [jb][face]
    int* s_cell = reinterpret_cast<int*>(xs + (size_t)jb_max * nf);
    int* s_sa = s_cell + nf;                          // side (+1 / -1) x 4 + normal axis
    __shared__ int start[kMaxI + 1];                  // per-column face ranges
    for (int q = threadIdx.x; q <= nI; q += blockDim.x) start[q] = nf;
    __syncthreads();
    for (int q = threadIdx.x; q < nf; q += blockDim.x) {
        const FaceInfo fi = faces[s.face_off + q];
        const int c = fi.col;
        if (q == 0 || faces[s.face_off + q - 1].col != c) start[c] = q;
        s_cell[q] = fi.cell;
        s_sa[q] = 4 * fi.s + fi.axis;
        s_tr[q] = face_tr[s.face_off + q];
        s_bst[q] = face_bst[s.face_off + q];
        s_be[q] = face_beta[s.face_off + q];
    }
    __syncthreads();
    // per basis, the data terms of its own two columns (g = 1 on the P-MBF,
    // g = -beta s on the U-MBF): sums over its faces in face order
    __shared__ double s_gsum[4][kMaxI];             // sum T_R, sum beta s T_R, sum beta^2 s^2 T_R, sum beta A_f
    for (int k = threadIdx.x; k < nI; k += blockDim.x) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        for (int q = start[k]; q < start[k + 1]; ++q) {
            const int sa = s_sa[q], ax = sa & 3;
            const double be = s_be[q];
            a0 += s_tr[q];
            a1 += s_bst[q];
            a2 += s_bst[q] * be * (double)((sa - ax) / 4);
            a3 += be * geo.area[ax];
        }
        s_gsum[0][k] = a0; s_gsum[1][k] = a1; s_gsum[2][k] = a2; s_gsum[3][k] = a3;
    }
    __syncthreads();
    const double* Xs = X + s.x_off;
    // The faces of basis k all carry column k; the Robin data g of MBF column j
    // on them is 1 (j = k, P-MBF), -beta s (j = nI + k, U-MBF) or 0, so the
    // traces are sum T_R x and sum beta s T_R x plus a correction on those two
    // columns: two FMAs per face and column, in four partial sums per trace
    // (face q0 + 4i + u of the basis to partial u; the partials are added in a
    // fixed order).  The face values of a column batch are gathered first by
    // consecutive threads over consecutive faces (neighbouring cells).
    for (int j0 = 0; j0 < m; j0 += jb_max) {
        const int jn = min(jb_max, m - j0);
        const int tot = jn * nf;
        for (int i0 = threadIdx.x; i0 < tot; i0 += 4 * blockDim.x) {
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {                 // four loads in flight, then the stores
                const int idx = i0 + u * blockDim.x;
                const int jb = idx / nf, q = idx - jb * nf;
                v[u] = idx < tot ? Xs[(long long)(j0 + jb) * N + s_cell[q]] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = i0 + u * blockDim.x;
                if (idx < tot) xs[idx] = v[u];
            }
        }
        __syncthreads();
        // S consecutive lanes per (basis, column) task when there are few tasks (large
        // whole-face bases): lane s takes the faces q0 + s + S i, four partial sums each,
        // combined in a fixed order (partials, then a butterfly over the S lanes)
        const int tasks = nI * jn;
        int S = 1;
        while (S < 32 && 2 * S * tasks <= (int)blockDim.x) S <<= 1;
        const int sub = threadIdx.x & (S - 1);
        for (int e0 = 0; e0 < tasks; e0 += blockDim.x / S) {
            const int e = e0 + threadIdx.x / S;
            const bool live = e < tasks;
            const int k = live ? e / jn : 0, jb = live ? e - k * jn : 0, j = j0 + jb;
            const int q0 = live ? start[k] : 0, q1 = live ? start[k + 1] : 0;
            const double* x = xs + (size_t)jb * nf;
            double pf[4] = {0.0, 0.0, 0.0, 0.0}, pu[4] = {0.0, 0.0, 0.0, 0.0};
            int q = q0 + sub;
            for (; q + 3 * S < q1; q += 4 * S) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    pf[u] = fma(s_tr[q + u * S], x[q + u * S], pf[u]);
                    pu[u] = fma(s_bst[q + u * S], x[q + u * S], pu[u]);
                }
            }
            for (int u = 0; q < q1; q += S, ++u) {
                pf[u] = fma(s_tr[q], x[q], pf[u]);
                pu[u] = fma(s_bst[q], x[q], pu[u]);
            }
            double sf = (pf[0] + pf[1]) + (pf[2] + pf[3]);
            double su = (pu[0] + pu[1]) + (pu[2] + pu[3]);
            for (int o = 1; o < S; o <<= 1) {             // the same sum in every lane of the group
                sf += __shfl_xor_sync(0xffffffffu, sf, o);
                su += __shfl_xor_sync(0xffffffffu, su, o);
            }
            if (!live || sub != 0) continue;
            double sdiag = 0.0;
            if (j == k) { sf -= s_gsum[0][k]; su -= s_gsum[1][k]; }               // g = 1
            else if (j == nI + k) {                                               // g = -beta s
                sf += s_gsum[1][k];
                su += s_gsum[2][k];
                sdiag = s_gsum[3][k];
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
        __syncthreads();                              // xs is refilled by the next batch
    }
}

__global__ void k_zero_int(int* p, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0;
}

__global__ void k_set_int(int* p, int v) { *p = v; }

// k_element: MBF columns per batch (at most 16, within about 96 KB of shared
// memory for the largest face set) and its dynamic shared memory (per face:
// cell, side and axis, three weights; the batch's face values)
constexpr size_t kElFaceBytes = 3 * sizeof(double) + 2 * sizeof(int);
static int element_batch(const Tables& t) {
    int mx = 1;
    for (const SubInfo& s : t.subs) mx = std::max(mx, s.nface);
    const long long room = 96 * 1024 - (long long)mx * (long long)kElFaceBytes;
    return (int)std::max(1LL, std::min(16LL, room / (long long)(mx * sizeof(double))));
}
static size_t element_smem(const Tables& t) {
    int mx = 1;
    for (const SubInfo& s : t.subs) mx = std::max(mx, s.nface);
    return (size_t)mx * kElFaceBytes + (size_t)element_batch(t) * mx * sizeof(double);
}

// ---------------------------------------------------------------------------
// Mean velocity post-processing (Eq. locprob_submean, the "Mean" method of the
// paper's two-phase section).  On every fine Gamma face the two sides'
// velocities are averaged, Ubar = (u^+ + u^-) / 2; every subdomain then
// re-solves its TPFA problem with Neumann data: Ubar on Gamma, the multiscale
// velocity on the walls.  The local matrix keeps the interior
// transmissibilities and loses the Robin and Dirichlet terms; the pure
// Neumann matrix is singular and the data compatible (the outward fluxes sum
// to the sources, Eq. weakcont_f), so the subdomain's last cell (slab order)
// is tied to pressure 0 by adding its own diagonal once more (exact for
// compatible data: the tie carries no flux).  The right-hand side goes into
// the particular column's Dirichlet slot: f V + rhs, rhs = -(prescribed
// outward fluxes).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_pp_coefficients(const SubInfo* __restrict__ subs, const double* __restrict__ u_in, Geo geo,
                  double* __restrict__ coef, double* __restrict__ scale, double* __restrict__ rhs_part,
                  long long nct) {
    const SubInfo s = subs[blockIdx.x];
    const long long ncells = (long long)geo.n[0] * geo.n[1] * geo.n[2];
    const long long stride[3] = {1, geo.n[0], (long long)geo.n[0] * geo.n[1]};
    int lstride[3];
    lstride[s.ua] = 1; lstride[s.va] = s.su; lstride[s.sa] = s.b;
    const double* tp[3];
    tp[s.ua] = coef + nct + s.cell_off;
    tp[s.va] = coef + 2 * nct + s.cell_off;
    tp[s.sa] = coef + 3 * nct + s.cell_off;
    for (int c = threadIdx.x; c < s.N; c += blockDim.x) {
        int lc[3];
        local_coords(s, c, lc);
        const long long g = global_cell(s, lc, geo.n);
        double d = 0.0, rd = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double* ulo = u_in + (long long)(2 * a) * ncells;
            const double* uhi = u_in + (long long)(2 * a + 1) * ncells;
            if (lc[a] + 1 < s.sz[a]) {
                d += tp[a][c];
            } else {                                     // box face on the +a side: Gamma (mean) or wall
                double v = uhi[g];
                if (s.o[a] + lc[a] + 1 < geo.n[a]) v = 0.5 * (v + ulo[g + stride[a]]);
                rd -= v * geo.area[a];
            }
            if (lc[a] > 0) {
                d += tp[a][c - lstride[a]];
            } else {                                     // box face on the -a side
                double v = ulo[g];
                if (s.o[a] + lc[a] > 0) v = 0.5 * (v + uhi[g - stride[a]]);
                rd += v * geo.area[a];
            }
        }
        if (c == s.N - 1) d += d > 0.0 ? d : 1.0;        // the tie
        const long long i = s.cell_off + c;
        coef[i] = d;
        scale[i] = f32_to_f64(rsqrtf(f64_to_f32_rz(d)));
        rhs_part[i] = rd;
    }
}

// Stop scale of the post-processing refinement: the Neumann systems of
// subdomains around a well have || |A||x| || up to 1e9 ||b|| (the oracle's
// sparse LU leaves a relative residual ~1e-7 there), so ||r|| <= tol ||b|| is
// out of FP64's reach.  After the first solve, the particular column's
// squared scale becomes sum_c (|b_c| + sum_k |a_ck x_k|)^2 (normwise
// Oettli-Prager form), and the sweeps stop on ||r|| <= tol times it.  One CTA
// per listed subdomain, fixed-order reduction.
__global__ void __launch_bounds__(kThreads)
k_pp_scale(const SubInfo* __restrict__ subs, const int* __restrict__ list, const double* __restrict__ coef,
           const double* __restrict__ rhs_part, const double* __restrict__ f, Geo geo, long long nct,
           const double* __restrict__ X, double* __restrict__ bnorm,
           const int* __restrict__ limit /* CTAs from *limit on have no subdomain; may be NULL */) {
    if (limit && (int)blockIdx.x >= *limit) return;
    const SubInfo s = subs[list[blockIdx.x]];
    const int N = s.N, b = s.b, su = s.su;
    const double* cd = coef + s.cell_off;
    const double* cu = coef + nct + s.cell_off;
    const double* cv = coef + 2 * nct + s.cell_off;
    const double* cs = coef + 3 * nct + s.cell_off;
    const double* x = X + s.x_off + (long long)(s.m - 1) * N;
    const double vol = geo.h[0] * geo.h[1] * geo.h[2];
    double acc = 0.0;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        int lc[3];
        local_coords(s, c, lc);
        const int i = c % b, u = i % su;
        double t = fabs(rhs_part[s.cell_off + c] + f[global_cell(s, lc, geo.n)] * vol) + fabs(cd[c] * x[c]);
        if (u + 1 < su) t += fabs(cu[c] * x[c + 1]);
        if (u > 0) t += fabs(cu[c - 1] * x[c - 1]);
        if (i + su < b) t += fabs(cv[c] * x[c + su]);
        if (i >= su) t += fabs(cv[c - su] * x[c - su]);
        if (c + b < N) t += fabs(cs[c] * x[c + b]);
        if (c >= b) t += fabs(cs[c - b] * x[c - b]);
        acc = fma(t, t, acc);
    }
    __shared__ double red[kThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) bnorm[s.rhs_off + s.m - 1] = fmin(red[0], 1e38);   // read back as FP32
}

// The subdomains of list[0 .. n) whose particular column did not converge, in
// any order (each keeps its own slots), and their count.
__global__ void k_pp_unconverged(const SubInfo* __restrict__ subs, const int* __restrict__ list, int n,
                                 const int* __restrict__ conv, int* __restrict__ out, int* __restrict__ count,
                                 int* __restrict__ total) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = list[i];
    const SubInfo s = subs[l];
    if (conv[s.rhs_off + s.m - 1] == 0) {
        out[atomicAdd(count, 1)] = l;
        atomicAdd(total, 1);
    }
}

// Post-processed velocity: TPFA of the Neumann solution (the particular column
// of the MBF array) on interior faces, Ubar on Gamma faces (both sides write the
// same value), the multiscale velocity on walls; then the per-cell mass balance
// sum(out-fluxes) - f V, reduced to its maximum (atomicMax on the bits of a
// non-negative double: order-independent).
__global__ void __launch_bounds__(kThreads)
k_pp_velocity(const SubInfo* __restrict__ subs, const double* __restrict__ X, const double* __restrict__ coef,
              const double* __restrict__ u_in, const double* __restrict__ f, Geo geo, long long nct,
              double* __restrict__ u_out, unsigned long long* __restrict__ mres_bits) {
    const SubInfo s = subs[blockIdx.x];
    const long long ncells = (long long)geo.n[0] * geo.n[1] * geo.n[2];
    const long long stride[3] = {1, geo.n[0], (long long)geo.n[0] * geo.n[1]};
    int lstride[3];
    lstride[s.ua] = 1; lstride[s.va] = s.su; lstride[s.sa] = s.b;
    const double* tp[3];
    tp[s.ua] = coef + nct + s.cell_off;
    tp[s.va] = coef + 2 * nct + s.cell_off;
    tp[s.sa] = coef + 3 * nct + s.cell_off;
    const double* pl = X + s.x_off + (long long)(s.m - 1) * s.N;
    double inv_area[3];
    for (int a = 0; a < 3; ++a) inv_area[a] = 1.0 / geo.area[a];
    for (int c = threadIdx.x; c < s.N; c += blockDim.x) {
        int lc[3];
        local_coords(s, c, lc);
        const long long g = global_cell(s, lc, geo.n);
        const double pc = pl[c];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double* ulo = u_in + (long long)(2 * a) * ncells;
            const double* uhi = u_in + (long long)(2 * a + 1) * ncells;
            double vhi, vlo;
            if (lc[a] + 1 < s.sz[a]) {
                vhi = tp[a][c] * (pc - pl[c + lstride[a]]) * inv_area[a];
            } else {
                vhi = uhi[g];
                if (s.o[a] + lc[a] + 1 < geo.n[a]) vhi = 0.5 * (vhi + ulo[g + stride[a]]);
            }
            if (lc[a] > 0) {
                vlo = tp[a][c - lstride[a]] * (pl[c - lstride[a]] - pc) * inv_area[a];
            } else {
                vlo = ulo[g];
                if (s.o[a] + lc[a] > 0) vlo = 0.5 * (vlo + uhi[g - stride[a]]);
            }
            u_out[(long long)(2 * a + 1) * ncells + g] = vhi;
            u_out[(long long)(2 * a) * ncells + g] = vlo;
        }
    }
    __syncthreads();                                      // this CTA wrote every face of its cells
    const double vol = geo.h[0] * geo.h[1] * geo.h[2];
    double mx = 0.0;
    for (int c = threadIdx.x; c < s.N; c += blockDim.x) {
        int lc[3];
        local_coords(s, c, lc);
        const long long g = global_cell(s, lc, geo.n);
        double div = -f[g] * vol;
        for (int a = 0; a < 3; ++a)
            div += (u_out[(long long)(2 * a + 1) * ncells + g] - u_out[(long long)(2 * a) * ncells + g]) * geo.area[a];
        mx = (div == div) ? fmax(mx, fabs(div)) : __longlong_as_double(0x7ff0000000000000LL);
    }
    __shared__ double red[kThreads];
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(mres_bits, (unsigned long long)__double_as_longlong(red[0]));
}

// FP64 fallback (mixed modes): after the last refinement sweep of a wave, every
// subdomain with a column still above the tolerance takes a slot (atomic
// ticket) whose record is a copy of its own with the block-factor and
// forward-value offsets moved into the fallback regions; the FP64 factor and
// solve kernels then run on the slots.  Which slot a subdomain gets does not
// change its result.  Subdomains without a slot (over the cap, or blocks the
// FP64 factor does not take) keep their mixed columns and count as
// unconverged.
__global__ void k_fb_collect(const SubInfo* __restrict__ subs, const int* __restrict__ list, int nlist,
                             const int* __restrict__ conv, int* __restrict__ status, SubInfo* __restrict__ fb_subs,
                             int* __restrict__ fb_list, int cap, long long wstride_slot, long long ystride_slot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nlist) return;
    SubInfo s = subs[list[i]];
    int bad = 0;
    for (int j = 0; j < s.m; ++j) bad += conv[s.rhs_off + j] == 0;
    if (!bad) return;
    int slot = -1;
    if (s.b <= kMaxBlock64) {
        slot = atomicAdd(&status[ST_FB_WAVE], 1);
        if (slot >= cap) slot = -1;
    }
    if (slot < 0) {
        atomicAdd(&status[ST_FB_LOST], 1);
        atomicAdd(&status[ST_UNCONVERGED], bad);
        return;
    }
    atomicAdd(&status[ST_FB_TOTAL], 1);
    s.w_off = (long long)slot * wstride_slot;
    s.y_off = (long long)slot * ystride_slot;
    fb_subs[slot] = s;
    fb_list[slot] = slot;
}

Geo make_geo(const mrcm_config& c) {
    Geo g;
    g.h[0] = c.hx; g.h[1] = c.hy; g.h[2] = c.hz;
    g.area[0] = c.hy * c.hz; g.area[1] = c.hx * c.hz; g.area[2] = c.hx * c.hy;
    g.n[0] = c.nx; g.n[1] = c.ny; g.n[2] = c.nz;
    return g;
}


}  // namespace

// Block factors of one wave's subdomains (register-resident FP32 kernel for
// b <= 64, packed shared-memory kernel otherwise; one launch per class).
int num_solve_variants() { return kNumSolveVariants; }

static void launch_factor_wave(const Tables& t, const DeviceTables& d, const Layout& L, char* ws, int precision,
                               int w, cudaStream_t st, Prof& P) {
    double* coef = (double*)(ws + L.coef);
    double* scale = (double*)(ws + L.scale);
    int* status = (int*)(ws + L.status);
    const int* wc = &t.wave_class_off[4 * w];
    const int o0 = wc[0], o1 = wc[1], o2 = wc[2], o3 = wc[3];
    const int n_small = o1 - o0, n_mid = o2 - o1, n_large = o3 - o2;
    if (precision == MRCM_FP64) {
        if (n_large > 0) {
            size_t sm = factor_smem<double>(std::min(t.max_b, kMaxBlock64));   // larger blocks: global slot
            MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor<double, false><<<n_large, kThreads, sm, st>>>(d.subs, d.class_list + o2, coef, scale,
                (double*)(ws + L.W), status, t.n_cells, (float*)(ws + L.scf), (float*)(ws + L.tsc), nullptr,
                (double*)(ws + L.big)));
        }
    } else {
        if (n_small > 0) {
            if (d.factor_variant == 0)
                MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor_reg<<<n_small, kRegMaxB, 0, st>>>(d.subs, d.class_list + o0, coef, scale,
                    (float*)(ws + L.W), status, t.n_cells, (float*)(ws + L.scf), (float*)(ws + L.tsc)));
            else if (d.factor_variant == 1)
                MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor_tile<8, 8><<<n_small, 64, 0, st>>>(d.subs, d.class_list + o0, coef, scale,
                    (float*)(ws + L.W), status, t.n_cells, (float*)(ws + L.scf), (float*)(ws + L.tsc)));
            else
                MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor_tile<4, 16><<<n_small, 256, 0, st>>>(d.subs, d.class_list + o0, coef, scale,
                    (float*)(ws + L.W), status, t.n_cells, (float*)(ws + L.scf), (float*)(ws + L.tsc)));
        }
        if (n_mid > 0) {
            if (d.factor_mid_variant == 1)       // tensor cores; its shared memory keeps <= 4 CTAs (4 x 128 TMEM columns) per SM
                MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor_tc<<<n_mid, kTcN, kTcSmem, st>>>(d.subs, d.class_list + o1, coef, scale,
                    (float*)(ws + L.W), status, t.n_cells, (float*)(ws + L.scf), (float*)(ws + L.tsc)));
            else
                MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor_tile<8, 16><<<n_mid, 256, 0, st>>>(d.subs, d.class_list + o1, coef, scale,
                    (float*)(ws + L.W), status, t.n_cells, (float*)(ws + L.scf), (float*)(ws + L.tsc)));
        }
        // the large class is ordered by b, largest first: one launch per run of
        // subdomains that share a thread count (packed kernel above kTriB)
        for (int q = o2; q < o3;) {
            const int nth = tri_threads(t.subs[t.class_list[q]].b);
            int e = q + 1;
            while (e < o3 && tri_threads(t.subs[t.class_list[e]].b) == nth) ++e;
            const int n = e - q;
            const int* lst = d.class_list + q;
            float* W = (float*)(ws + L.W);
            float* scf = (float*)(ws + L.scf);
            float* tsc = (float*)(ws + L.tsc);
            switch (nth) {
            case 192: MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor_tri<192><<<n, 192, 0, st>>>(d.subs, lst, coef, scale, W, status, t.n_cells, scf, tsc)); break;
            case 320: MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor_tri<320><<<n, 320, 0, st>>>(d.subs, lst, coef, scale, W, status, t.n_cells, scf, tsc)); break;
            case 512: MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor_tri<512><<<n, 512, 0, st>>>(d.subs, lst, coef, scale, W, status, t.n_cells, scf, tsc)); break;
            case 544: MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor_tri<544><<<n, 544, 0, st>>>(d.subs, lst, coef, scale, W, status, t.n_cells, scf, tsc)); break;
            default: {
                size_t sm = factor_smem<float>(t.max_b);
                MRCM_LAUNCH(P, "k_block_factor", st, k_block_factor<float, true><<<n, kThreads, sm, st>>>(d.subs, lst, coef, scale, W, status, t.n_cells, scf, tsc, nullptr, nullptr));
            }
            }
            q = e;
        }
    }
}

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
                                             (double*)(ws + L.face_beta), (double*)(ws + L.face_u),
                                             (double*)(ws + L.face_bst), t.n_cells));
    // the learned form solves the local problems iteratively: coefficients only
    if (t.n_waves == 1 && precision != MRCM_LEARNED_PCG) launch_factor_wave(t, d, L, ws, precision, 0, st, P);
    return (int)cudaGetLastError();
}

static size_t solve_smem_bytes(const Tables& t, int precision) {
    const int mpad = (t.max_m + 3) & ~3;
    size_t sm = 0;
    for (const SubInfo& sb : t.subs)
        sm = std::max(sm, precision == MRCM_FP64 ? solve_smem_layout<double>(sb.b, mpad, sb.N).total
                                                 : solve_smem_layout<float>(sb.b, mpad, sb.N).total);
    return sm + 16;                                // + the two mbarriers, after the largest layout
}

// One-time kernel configuration (dynamic shared memory limits, persistent
// grid sizes); runs outside any stream capture.
int configure_local(const Tables& t, DeviceTables& d) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    const bool f64 = t.cfg.precision == MRCM_FP64;
    cudaFuncSetAttribute(k_element, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)element_smem(t));
    d.solve_smem = solve_smem_bytes(t, t.cfg.precision);
    for (int v = 0; v < kNumSolveVariants; ++v) {
        const void* k0 = f64 ? solve_kernel<double, false, false>(v) : solve_kernel<float, true, false>(v);
        const void* k1 = f64 ? solve_kernel<double, false, true>(v) : solve_kernel<float, true, true>(v);
        cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.solve_smem);
        cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.solve_smem);
        int occ0 = 0, occ1 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, k0, variant_threads(v), d.solve_smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, k1, variant_threads(v), d.solve_smem);
        d.solve_occ[v] = std::max(1, occ0);
        d.sweep_occ[v] = std::max(1, occ1);
    }
    if (!f64) {
        // the FP64 solve kernels of the mixed modes' fallback and post-processing (variant 0)
        const int mpad = (t.max_m + 3) & ~3;
        size_t sm = 0;
        for (const SubInfo& sb : t.subs)
            if (sb.b <= kMaxBlock64) sm = std::max(sm, solve_smem_layout<double>(sb.b, mpad, sb.N).total);
        d.f64_solve_smem = sm + 16;
        const void* k0 = solve_kernel<double, false, false>(0);
        const void* k1 = solve_kernel<double, false, true>(0);
        cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.f64_solve_smem);
        cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.f64_solve_smem);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k1, variant_threads(0), d.f64_solve_smem);
        d.f64_occ = std::max(1, occ);
    }
    cudaFuncSetAttribute(k_block_factor<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)factor_smem<double>(std::min(t.max_b, kMaxBlock64)));
    cudaFuncSetAttribute(k_block_factor<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)factor_smem<float>(t.max_b));
    cudaFuncSetAttribute(k_block_factor_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    return (int)cudaGetLastError();
}

static LocalArgs local_args(const Tables& t, const DeviceTables& d, const Layout& L, char* ws, const double* f) {
    LocalArgs g;
    g.subs = d.subs; g.faces = d.faces;
    g.coef = (const double*)(ws + L.coef); g.scale = (const double*)(ws + L.scale);
    g.scf = (const float*)(ws + L.scf); g.tsc = (const float*)(ws + L.tsc);
    g.face_tr = (const double*)(ws + L.face_tr); g.face_beta = (const double*)(ws + L.face_beta);
    g.face_u = (const double*)(ws + L.face_u);
    g.rhs_dir = (const double*)(ws + L.rhs_part); g.f = f; g.geo = make_geo(t.cfg); g.nct = t.n_cells;
    g.X = (double*)(ws + L.X); g.Ybuf = (void*)(ws + L.R);
    g.conv = (int*)(ws + L.conv); g.bnorm = (double*)(ws + L.colnorm);
    g.tol2 = 0.0; g.status = (int*)(ws + L.status);
    g.mpad = (t.max_m + 3) & ~3;
    g.list = d.solve_list; g.nlist = (int)t.subs.size();
    g.queue = (int*)(ws + L.status) + ST_QUEUE;
    g.count_unconverged = 0;
    g.bar_off = (int)d.solve_smem - 16;
    g.last_only = 0;
    g.nlist_dev = nullptr;
    g.col_groups = 1;
    g.passes = 1;
    return g;
}

// Launch one local-solve pass (first solve or refinement sweep) with variant v.
static void launch_local_pass(const Tables& t, const DeviceTables& d, LocalArgs& g, const void* W, bool sweep,
                              int v, cudaStream_t st, Prof& P) {
    const bool f64 = t.cfg.precision == MRCM_FP64;
    const void* k = f64 ? (sweep ? solve_kernel<double, false, true>(v) : solve_kernel<double, false, false>(v))
                        : (sweep ? solve_kernel<float, true, true>(v) : solve_kernel<float, true, false>(v));
    const int occ = sweep ? d.sweep_occ[v] : d.solve_occ[v];
    const int grid = std::max(1, std::min(g.nlist, d.sms * occ));
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(g.queue, 0));
    void* args[] = {(void*)&g, (void*)&W};
    MRCM_LAUNCH(P, sweep ? "k_ir_sweep" : "k_local_solve", st,
                cudaLaunchKernel(k, dim3(grid), dim3(variant_threads(v)), args, d.solve_smem, st));
}

// FP64 fallback of one wave (see k_fb_collect): slots, FP64 block factors of
// the slots, FP64 solve of all their columns (replacing the mixed ones).
constexpr int kFbGroups = 4;
constexpr int kPpMixedSweeps = 10;         // FP64 refinement sweeps of the post-processing's FP32 pass
constexpr double kPpMixedTol = 1e-13;      // and their stop on the backward error: the post-processed
                                           // velocity must balance mass to about FP64 level

static void launch_fallback(const Tables& t, const DeviceTables& d, const Layout& L, char* ws, const LocalArgs& g0,
                            int cap, long long wstride_slot, long long ystride_slot, cudaStream_t st, Prof& P) {
    int* status = (int*)(ws + L.status);
    SubInfo* fb_subs = (SubInfo*)(ws + L.fb_subs);
    int* fb_list = (int*)(ws + L.fb_list);
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_FB_WAVE, 0));
    MRCM_LAUNCH(P, "k_fb_collect", st, k_fb_collect<<<(g0.nlist + 127) / 128, 128, 0, st>>>(d.subs, g0.list, g0.nlist,
                g0.conv, status, fb_subs, fb_list, cap, wstride_slot, ystride_slot));
    int bmax = 0;
    for (const SubInfo& s : t.subs) if (s.b <= kMaxBlock64) bmax = std::max(bmax, s.b);
    MRCM_LAUNCH(P, "k_fb_factor", st, k_block_factor<double, false><<<cap, kThreads, factor_smem<double>(bmax), st>>>(
                fb_subs, fb_list, g0.coef, g0.scale, (double*)(ws + L.fb_W), status, t.n_cells, nullptr, nullptr,
                status + ST_FB_WAVE, nullptr));
    LocalArgs g = g0;
    g.subs = fb_subs;
    g.list = fb_list;
    g.nlist = cap;
    g.nlist_dev = status + ST_FB_WAVE;
    g.Ybuf = (void*)(ws + L.fb_Y);
    g.last_only = 0;
    g.bar_off = (int)d.f64_solve_smem - 16;
    g.count_unconverged = 0;
    // a few fallback subdomains would leave most SMs idle on a long FP64 chain: up to
    // kFbGroups CTAs share each one, split by columns
    g.col_groups = kFbGroups;
    const int grid = std::max(1, std::min(cap * kFbGroups, d.sms * d.f64_occ));
    const void* Wfb = (const void*)(ws + L.fb_W);
    void* args[] = {(void*)&g, (void*)&Wfb};
    // the FP64 form's solve: direct solve through the FP64 block inverses, then one FP64 refinement step
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(g.queue, 0));
    MRCM_LAUNCH(P, "k_fb_solve", st, cudaLaunchKernel(solve_kernel<double, false, false>(0), dim3(grid),
                dim3(variant_threads(0)), args, d.f64_solve_smem, st));
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(g.queue, 0));
    MRCM_LAUNCH(P, "k_fb_solve", st, cudaLaunchKernel(solve_kernel<double, false, true>(0), dim3(grid),
                dim3(variant_threads(0)), args, d.f64_solve_smem, st));
}

int launch_solve_mbf(const Tables& t, const DeviceTables& d, const Layout& L, char* ws,
                     const double* f, int precision, int sweeps, double tol, void* stream, Prof& P) {
    cudaStream_t st = (cudaStream_t)stream;
    const int nsub = (int)t.subs.size();
    int* status = (int*)(ws + L.status);
    LocalArgs g = local_args(t, d, L, ws, f);
    g.tol2 = tol * tol;
    const void* W = (const void*)(ws + L.W);
    int fb_cap = 0;
    long long fb_stride = 0, fb_ystride = 0;
    fallback_params(t, &fb_cap, &fb_stride, &fb_ystride);
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_UNCONVERGED, 0));
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_FB_TOTAL, 0));
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_FB_LOST, 0));
    for (int w = 0; w < t.n_waves; ++w) {
        // one memory-bounded wave: factor (when waves share the W region), solve, refine
        if (t.n_waves > 1) launch_factor_wave(t, d, L, ws, precision, w, st, P);
        g.list = d.solve_list + t.wave_off[w];
        g.nlist = t.wave_off[w + 1] - t.wave_off[w];
        g.count_unconverged = 0;
        launch_local_pass(t, d, g, W, false, d.solve_variant, st, P);
        if (precision != MRCM_FP64) {
            // all sweeps in one launch, each subdomain's back to back (a subdomain that needs more
            // sweeps than most no longer holds up a launch of its own per sweep), or one launch per
            // sweep when the autotuner measured that faster (uneven subdomain sizes)
            for (int it = 0; it < sweeps;) {
                const int np = d.sweeps_separate ? 1 : sweeps - it;
                g.passes = np;
                g.count_unconverged = it + np == sweeps && fb_cap == 0 ? 1 : 0;
                launch_local_pass(t, d, g, W, true, d.sweep_variant, st, P);
                it += np;
            }
            g.passes = 1;
            if (fb_cap > 0) launch_fallback(t, d, L, ws, g, fb_cap, fb_stride, fb_ystride, st, P);
        } else {
            // FP64 form: the direct solve through the explicit block inverses plus one
            // FP64 refinement step (the same residual sweep), for FP64-level MBFs
            g.count_unconverged = 0;
            launch_local_pass(t, d, g, W, true, d.sweep_variant, st, P);
        }
    }
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_SWEEPS, precision == MRCM_FP64 ? 1 : sweeps));
    MRCM_LAUNCH(P, "k_element", st, k_element<<<nsub, kThreads, element_smem(t), st>>>(d.subs, d.faces, (double*)(ws + L.face_tr), (double*)(ws + L.face_beta),
                                        (const double*)(ws + L.face_bst),
                                        (const double*)(ws + L.X), g.geo, (double*)(ws + L.elem), (double*)(ws + L.elem_b),
                                        element_batch(t)));
    return (int)cudaGetLastError();
}

// Mean velocity post-processing: Neumann coefficients and right-hand sides
// from the multiscale velocity, then per wave the block factor of the Neumann
// matrices and the solve of the one (particular) column, refined like the
// MBF columns in mixed precision; then the post-processed velocity.  Leaves
// the local coefficients, factors and MBF array overwritten.
int launch_postprocess(const Tables& t, const DeviceTables& d, const Layout& L, char* ws, const double* u,
                       double* u_out, double* mres, const double* f, int precision, int sweeps, double tol,
                       void* stream, Prof& P) {
    cudaStream_t st = (cudaStream_t)stream;
    const int nsub = (int)t.subs.size();
    int* status = (int*)(ws + L.status);
    double* coef = (double*)(ws + L.coef);
    const Geo geo = make_geo(t.cfg);
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_UNCONVERGED, 0));
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_FB_TOTAL, 0));
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_FB_LOST, 0));
    MRCM_LAUNCH(P, "k_pp_coefficients", st, k_pp_coefficients<<<nsub, kThreads, 0, st>>>(d.subs, u, geo, coef,
                (double*)(ws + L.scale), (double*)(ws + L.rhs_part), t.n_cells));
    LocalArgs g = local_args(t, d, L, ws, f);
    g.tol2 = tol * tol;
    g.last_only = 1;
    const void* W = (const void*)(ws + L.W);
    if (precision == MRCM_FP64) {
        for (int w = 0; w < t.n_waves; ++w) {
            launch_factor_wave(t, d, L, ws, precision, w, st, P);
            g.list = d.solve_list + t.wave_off[w];
            g.nlist = t.wave_off[w + 1] - t.wave_off[w];
            g.count_unconverged = 0;
            launch_local_pass(t, d, g, W, false, d.solve_variant, st, P);
            MRCM_LAUNCH(P, "k_pp_scale", st, k_pp_scale<<<g.nlist, kThreads, 0, st>>>(g.subs, g.list, coef, g.rhs_dir,
                        f, geo, t.n_cells, g.X, g.bnorm, nullptr));
            for (int it = 0; it < sweeps; ++it) {
                g.count_unconverged = it + 1 == sweeps ? 1 : 0;
                launch_local_pass(t, d, g, W, true, d.sweep_variant, st, P);
            }
        }
    } else {
        // (1) every subdomain: FP32 block factors of the tied Neumann matrix, the FP32 solve
        // of the one column and kPpMixedSweeps FP64 refinement sweeps in one launch (stop on
        // the backward error, kPpMixedTol); most subdomains converge
        for (int w = 0; w < t.n_waves; ++w) {
            launch_factor_wave(t, d, L, ws, precision, w, st, P);
            g.list = d.solve_list + t.wave_off[w];
            g.nlist = t.wave_off[w + 1] - t.wave_off[w];
            g.count_unconverged = 0;
            launch_local_pass(t, d, g, W, false, d.solve_variant, st, P);
            MRCM_LAUNCH(P, "k_pp_scale", st, k_pp_scale<<<g.nlist, kThreads, 0, st>>>(g.subs, g.list, coef, g.rhs_dir,
                        f, geo, t.n_cells, g.X, g.bnorm, nullptr));
            g.passes = kPpMixedSweeps;
            g.tol2 = kPpMixedTol * kPpMixedTol;
            launch_local_pass(t, d, g, W, true, d.sweep_variant, st, P);
            g.passes = 1;
            g.tol2 = tol * tol;
        }
        // (2) the tied Neumann blocks too ill-conditioned for that: FP64 block factors in the W
        // region (post-processing waves), FP64 solve and refinement of the one column.  A
        // non-positive FP32 pivot of (1) only marks a block for this stage (its column then does
        // not converge): the count restarts for the FP64 factors.
        MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_NOT_SPD, 0));
        g.subs = d.pp_subs;
        g.bar_off = (int)d.f64_solve_smem - 16;
        const int nw = (int)t.pp_wave_off.size() - 1;
        int bmax = 0;
        for (const SubInfo& s : t.subs) bmax = std::max(bmax, s.b);
        int* plist = (int*)(ws + L.pp_list);
        int* cnt = status + ST_FB_WAVE;
        g.list = plist;
        g.nlist_dev = cnt;
        for (int w = 0; w < nw; ++w) {
            const int n = t.pp_wave_off[w + 1] - t.pp_wave_off[w];
            g.nlist = n;
            MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(cnt, 0));
            MRCM_LAUNCH(P, "k_pp_unconverged", st, k_pp_unconverged<<<(n + 127) / 128, 128, 0, st>>>(d.subs,
                        d.solve_list + t.pp_wave_off[w], n, g.conv, plist, cnt, status + ST_FB_TOTAL));
            MRCM_LAUNCH(P, "k_pp_factor", st, k_block_factor<double, false><<<n, kThreads, factor_smem<double>(bmax), st>>>(
                        d.pp_subs, plist, coef, (const double*)(ws + L.scale), (double*)(ws + L.W), status, t.n_cells,
                        nullptr, nullptr, cnt, nullptr));
            const int grid = std::max(1, std::min(n, d.sms * d.f64_occ));
            void* args[] = {(void*)&g, (void*)&W};
            g.count_unconverged = 0;
            MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(g.queue, 0));
            MRCM_LAUNCH(P, "k_pp_solve", st, cudaLaunchKernel(solve_kernel<double, false, false>(0), dim3(grid),
                        dim3(variant_threads(0)), args, d.f64_solve_smem, st));
            MRCM_LAUNCH(P, "k_pp_scale", st, k_pp_scale<<<n, kThreads, 0, st>>>(g.subs, plist, coef, g.rhs_dir,
                        f, geo, t.n_cells, g.X, g.bnorm, cnt));
            for (int it = 0; it < sweeps; ++it) {
                g.count_unconverged = it + 1 == sweeps ? 1 : 0;
                MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(g.queue, 0));
                MRCM_LAUNCH(P, "k_pp_solve", st, cudaLaunchKernel(solve_kernel<double, false, true>(0), dim3(grid),
                            dim3(variant_threads(0)), args, d.f64_solve_smem, st));
            }
        }
        g.nlist_dev = nullptr;
    }
    double* psum = (double*)(ws + L.psum);
    unsigned long long* mbits = (unsigned long long*)(psum + nsub + 1);
    MRCM_LAUNCH(P, "k_zero_int", st, k_zero_int<<<1, 32, 0, st>>>((int*)mbits, 2));
    MRCM_LAUNCH(P, "k_pp_velocity", st, k_pp_velocity<<<nsub, kThreads, 0, st>>>(d.subs, (const double*)(ws + L.X), coef, u,
                f, geo, t.n_cells, u_out, mbits));
    if (mres) cudaMemcpyAsync(mres, mbits, sizeof(double), cudaMemcpyDeviceToDevice, st);
    return (int)cudaGetLastError();
}

// After the learned form's column solves (which leave conv[] = 1 on the
// columns within the tolerance): the FP64 direct fallback of every subdomain
// with a column that is not, then the traces of all columns.
int launch_local_finish(const Tables& t, const DeviceTables& d, const Layout& L, char* ws, const double* f,
                        void* stream, Prof& P) {
    cudaStream_t st = (cudaStream_t)stream;
    int* status = (int*)(ws + L.status);
    const int nsub = (int)t.subs.size();
    LocalArgs g = local_args(t, d, L, ws, f);
    int fb_cap = 0;
    long long fb_stride = 0, fb_ystride = 0;
    fallback_params(t, &fb_cap, &fb_stride, &fb_ystride);
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_FB_TOTAL, 0));
    MRCM_LAUNCH(P, "k_set_int", st, k_set_int<<<1, 1, 0, st>>>(status + ST_FB_LOST, 0));
    if (fb_cap > 0) {
        // in chunks of fb_cap subdomains of the cost-ordered list: each chunk's slots are reused
        for (int q = 0; q < nsub; q += fb_cap) {
            LocalArgs gq = g;
            gq.list = d.solve_list + q;
            gq.nlist = std::min(fb_cap, nsub - q);
            launch_fallback(t, d, L, ws, gq, fb_cap, fb_stride, fb_ystride, st, P);
        }
    } else {
        // no fallback: the columns that did not converge are counted (no slot is taken)
        MRCM_LAUNCH(P, "k_fb_collect", st, k_fb_collect<<<(nsub + 127) / 128, 128, 0, st>>>(d.subs, d.solve_list, nsub,
                    g.conv, status, (SubInfo*)(ws + L.fb_subs), (int*)(ws + L.fb_list), 0, 0, 0));
    }
    MRCM_LAUNCH(P, "k_element", st, k_element<<<nsub, kThreads, element_smem(t), st>>>(d.subs, d.faces, (double*)(ws + L.face_tr), (double*)(ws + L.face_beta),
                                        (const double*)(ws + L.face_bst),
                                        (const double*)(ws + L.X), g.geo, (double*)(ws + L.elem), (double*)(ws + L.elem_b),
                                        element_batch(t)));
    return (int)cudaGetLastError();
}

// Autotuner: (0) time the factor kernels for blocks with b <= 64 and keep
// the faster (the factor is then recomputed with it); (1) time every variant's first solve (median of `reps`) and keep
// the fastest; (2) for every variant, after an untimed first solve, time the
// whole refinement sequence as the solve runs it (ir_max_sweeps sweeps with
// the configured tolerance, so retired columns shrink the later sweeps) and
// keep the fastest.  Tuned on the first wave.
int autotune_local(const Tables& t, DeviceTables& d, const Layout& L, char* ws, const double* f,
                   void* stream, int reps, int* best_solve, int* best_sweep, int* best_factor, int* best_factor_mid,
                   float* ms_out) {
    cudaStream_t st = (cudaStream_t)stream;
    LocalArgs g = local_args(t, d, L, ws, f);
    g.tol2 = t.cfg.ir_tol * t.cfg.ir_tol;
    const void* W = (const void*)(ws + L.W);
    Prof dummy;
    g.list = d.solve_list;                      // tune on the first wave
    g.nlist = t.wave_off[1];
    if (t.n_waves > 1) launch_factor_wave(t, d, L, ws, t.cfg.precision, 0, st, dummy);
    const bool mixed = t.cfg.precision != MRCM_FP64;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto median = [](std::vector<float>& v) { std::sort(v.begin(), v.end()); return v[v.size() / 2]; };
    // (0) factor kernel for the blocks with b <= 64 (mixed precision): a row per thread, 8 x 8 or 4 x 4 tiles
    if (mixed && t.wave_class_off[1] > t.wave_class_off[0]) {
        float bestf = 1e30f;
        for (int fv = 0; fv < kNumFactorVariants; ++fv) {
            d.factor_variant = fv;
            std::vector<float> tf;
            for (int r = 0; r < reps; ++r) {
                cudaEventRecord(e0, st);
                launch_factor_wave(t, d, L, ws, t.cfg.precision, 0, st, dummy);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                tf.push_back(ms);
            }
            const float mf = median(tf);
            if (mf < bestf) { bestf = mf; *best_factor = fv; }
        }
        d.factor_variant = *best_factor;
        launch_factor_wave(t, d, L, ws, t.cfg.precision, 0, st, dummy);
    }
    // (0b) factor kernel for 64 < b <= 128: register tiles or the tensor-core (TMEM) kernel.  The
    // tensor-core factor must also keep the refinement converging: its wave-0 solve may leave at
    // most 1.5x (+16) the unconverged columns of the register-tile factor after the configured sweeps.
    if (mixed && t.wave_class_off[2] > t.wave_class_off[1]) {
        float bestf = 1e30f;
        int unconv[2] = {0, 0};
        int* status = (int*)(ws + L.status);
        for (int fv = 0; fv < 2; ++fv) {
            d.factor_mid_variant = fv;
            std::vector<float> tf;
            for (int r = 0; r < reps; ++r) {
                cudaEventRecord(e0, st);
                launch_factor_wave(t, d, L, ws, t.cfg.precision, 0, st, dummy);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                tf.push_back(ms);
            }
            // convergence of the refinement with this factor (wave 0)
            k_set_int<<<1, 1, 0, st>>>(status + ST_UNCONVERGED, 0);
            launch_local_pass(t, d, g, W, false, d.solve_variant, st, dummy);
            for (int it = 0; it < t.cfg.ir_max_sweeps; ++it) {
                g.count_unconverged = it + 1 == t.cfg.ir_max_sweeps ? 1 : 0;
                launch_local_pass(t, d, g, W, true, d.sweep_variant, st, dummy);
            }
            g.count_unconverged = 0;
            cudaMemcpyAsync(&unconv[fv], status + ST_UNCONVERGED, sizeof(int), cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            const float mf = median(tf);
            const bool converges = fv == 0 || unconv[fv] <= unconv[0] + unconv[0] / 2 + 16;
            if (converges && mf < bestf) { bestf = mf; *best_factor_mid = fv; }
        }
        d.factor_mid_variant = *best_factor_mid;
        launch_factor_wave(t, d, L, ws, t.cfg.precision, 0, st, dummy);
    }
    float best0 = 1e30f, best1 = 1e30f;
    *best_solve = 0;
    *best_sweep = 0;
    for (int v = 0; v < kNumSolveVariants; ++v) {
        std::vector<float> t0;
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(e0, st);
            launch_local_pass(t, d, g, W, false, v, st, dummy);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t0.push_back(ms);
        }
        const float m0 = median(t0);
        if (ms_out) ms_out[2 * v] = m0;
        if (m0 < best0) { best0 = m0; *best_solve = v; }
    }
    if (mixed) {
        for (int v = 0; v < kNumSolveVariants; ++v) {
            std::vector<float> t1;
            for (int r = 0; r < reps; ++r) {
                launch_local_pass(t, d, g, W, false, *best_solve, st, dummy);
                cudaEventRecord(e0, st);
                g.passes = t.cfg.ir_max_sweeps;          // all sweeps in one launch
                if (g.passes > 0) launch_local_pass(t, d, g, W, true, v, st, dummy);
                g.passes = 1;
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                t1.push_back(ms);
            }
            const float m1 = median(t1);
            if (ms_out) ms_out[2 * v + 1] = m1;
            if (m1 < best1) { best1 = m1; *best_sweep = v; }
        }
        // the chosen variant with one launch per sweep
        std::vector<float> t2;
        for (int r = 0; r < reps && t.cfg.ir_max_sweeps > 0; ++r) {
            launch_local_pass(t, d, g, W, false, *best_solve, st, dummy);
            cudaEventRecord(e0, st);
            for (int it = 0; it < t.cfg.ir_max_sweeps; ++it) launch_local_pass(t, d, g, W, true, *best_sweep, st, dummy);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t2.push_back(ms);
        }
        d.sweeps_separate_ms = t2.empty() ? -1.0f : median(t2);
        d.sweeps_separate = (!t2.empty() && d.sweeps_separate_ms < best1) ? 1 : 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (int)cudaGetLastError();
}

}  // namespace mrcm
