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
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "mrcm_devmath.cuh"
#include "mrcm_internal.h"

namespace mrcm {

namespace {

constexpr int kThreads = 256;

// Programmatic dependent launch: the kernels of the interface stage are
// launched with programmatic stream serialization, so each can be scheduled
// while its predecessor on the stream finishes; it waits here until the
// predecessor has completed and its writes are visible.
__device__ __forceinline__ void pdl_begin() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
constexpr int kPanel = 32;        // LDL^T panel width
constexpr int kTile = 64;         // assembly tile

__global__ void k_assemble_csr(int nrows, const int* __restrict__ rowptr, const long long* __restrict__ src_lo,
                               const long long* __restrict__ src_hi, const int* __restrict__ rsl,
                               const int* __restrict__ rsh, const int* __restrict__ colidx,
                               const double* __restrict__ elem, const double* __restrict__ elem_b,
                               double* __restrict__ val, double* __restrict__ b, double* __restrict__ dscale,
                               int pin) {
    pdl_begin();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    double diag = 0.0, rowmax = 0.0;
    for (int q = rowptr[r]; q < rowptr[r + 1]; ++q) {
        double v = 0.0;
        if (src_lo[q] >= 0) v += elem[src_lo[q]];
        if (src_hi[q] >= 0) v += elem[src_hi[q]];
        val[q] = v;
        if (colidx[q] == r) diag = v;
        rowmax = fmax(rowmax, fabs(v));
    }
    b[r] = elem_b[rsl[r]] + elem_b[rsh[r]];
    double ad = fabs(diag);
    // The pressure constant is removed by -c e_0 e_0^T with c = 1 / dscale[0]^2 (the factorisation
    // subtracts 1 from the scaled pinned entry); any c > 0 gives the solution with pi^p_0 = 0.  c is
    // the row's largest entry: |A_00| itself unless A_00 vanishes, which it does when the
    // subdomains around basis 0 carry no other basis (their P-MBF is the constant 1, no flux).
    if (pin && r == 0) ad = rowmax;
    dscale[r] = ad > 0.0 ? rsqrt(ad) : 1.0;
}

__device__ __forceinline__ double dof_sign(int dof, int NV) { return dof < NV ? 1.0 : -1.0; }


// LDL^T of the nbk x nbk (nbk <= 32) diagonal block of a front, in place
// (strict lower part becomes L11, the diagonal D), together with V = L11^{-1}.
// Row i of the work array T holds [row i of the block, both triangles | row i
// of V]; V starts as I.  Step k: with the multipliers w_c = T[k][c] / d_k on
// the block part (k < c) and w_c = V[k][c] / d_k on the V part (c <= k), every
// row i > k takes
//   T[i][c] -= T[i][k] w_c   (every block column c > k and every c <= k of V),
// the rank-1 Schur update of the block and V <- (I - l e_k^T) V at once (row k
// of V is final at step k).  Block column k is not written after step k - 1,
// so L = T[i][k] / d_k is formed once at the end: one barrier per pivot.  One
// lane per column: a row costs one FP64 FMA per step.  Warp 0 updates row
// k + 1 alone; its lane k + 1 computes 1 / d_{k+1} (one cubic Newton step)
// from the fresh diagonal, and the warp forms the next step's multipliers
// from the row it holds (the upper triangle is kept for that) into one of two
// shared vectors, so the other warps, which update the remaining rows, read
// them instead of each forming them.  A zero or NaN pivot is replaced by 1
// and counted.  Block-wide, >= 2 warps.
constexpr int kDiagW = 2 * kPanel + 1;

// v == 0 or NaN, from the bits (integer operations: an FP64 compare would add
// an FP64-unit latency to the pivot chain).
__device__ __forceinline__ bool zero_or_nan(double v) {
    const unsigned long long m = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    return m == 0ull || m > 0x7FF0000000000000ull;
}

constexpr int kDiagWork = kPanel * kDiagW + 3 * kPanel + 4;   // doubles of shared work space
__device__ void factor_diag_block(double* __restrict__ A, int n, int k0, int nbk, double* __restrict__ Pinv,
                                  int* status, double* work) {
    double (*T)[kDiagW] = reinterpret_cast<double (*)[kDiagW]>(work);
    double* sinv = work + kPanel * kDiagW;                    // 1 / d_k for every k
    double* swc = sinv + kPanel;                              // multipliers of step k at swc[(k & 1) * kPanel]
    int* zero = reinterpret_cast<int*>(swc + 2 * kPanel);
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nthr >> 5;
    __syncthreads();                                          // the block's last writes are complete
    for (int e = tid; e < kPanel * 2 * kPanel; e += nthr) {
        const int i = e >> 6, c = e & 63;
        double v;
        if (c < kPanel) v = (i < nbk && c < nbk) ? A[(long long)(k0 + max(i, c)) * n + k0 + min(i, c)] : 0.0;
        else v = (c - kPanel == i) ? 1.0 : 0.0;
        T[i][c] = v;
    }
    __syncthreads();
    if (w == 0) {                                             // the first pivot and its multipliers
        double d = T[0][0];
        const bool z = zero_or_nan(d);
        if (z) d = 1.0;
        const double inv0 = rcp64c(d);
        swc[lane] = (lane == 0 ? 1.0 : T[0][lane]) * inv0;
        if (lane == 0) {
            *zero = z ? 1 : 0;
            if (z) T[0][0] = 1.0;
            sinv[0] = inv0;
        }
    }
    for (int k = 0; k < nbk; ++k) {
        __syncthreads();                                      // rows of step k - 1 done, multipliers of step k ready
        const int c = lane;
        const bool vpart = c <= k;
        if (k + 1 + (w == 0 ? 0 : w) >= nbk) continue;        // no row for this warp at this step
        const double wc = swc[(k & 1) * kPanel + c];
        if (w == 0) {
            const int i = k + 1;
            double* dst = vpart ? &T[i][kPanel + c] : &T[i][c];
            double v = fma(-T[i][k], wc, *dst);
            double inv = 0.0;
            if (c == i) {                                     // the next pivot, straight from the register
                if (zero_or_nan(v)) { v = 1.0; *zero = 1; }
                inv = rcp64c(v);
                sinv[i] = inv;
            }
            *dst = v;
            inv = __shfl_sync(0xffffffffu, inv, i);
            swc[((k + 1) & 1) * kPanel + c] = (c == i ? 1.0 : v) * inv;
        } else {
            for (int i = k + 1 + w; i < nbk; i += nw - 1) {
                double* dst = vpart ? &T[i][kPanel + c] : &T[i][c];
                *dst = fma(-T[i][k], wc, *dst);
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < kPanel * kPanel; e += nthr) {
        const int i = e >> 5, c = e & 31;
        if (i < nbk && c <= i) A[(long long)(k0 + i) * n + k0 + c] = c == i ? T[i][i] : T[i][c] * sinv[c];
        Pinv[e] = T[i][kPanel + c];
    }
    if (tid == 0 && *zero) atomicAdd(&status[ST_ZERO_PIVOT], 1);
}

// Front assembly as a gather: every lower-triangle entry (r >= q) of the
// front is written once, as the sum (child 0 first) of the children's
// entries at the same dofs -- J-signed, scaled subdomain blocks for leaves,
// the lower triangle of the Schur complement otherwise.  64x64 tiles of the
// lower triangle are spread over the grid; blockIdx.y selects the front.
__global__ void __launch_bounds__(kThreads)
k_front_assemble(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids,
                 const int* __restrict__ inv, const int* __restrict__ dofs, const SubInfo* __restrict__ subs,
                 const double* __restrict__ elem, const double* __restrict__ dscale, int NV,
                 double* __restrict__ F, double* __restrict__ P, int* __restrict__ status) {
    pdl_begin();
    const FrontInfo fr = fronts[ids[blockIdx.y]];
    const int n = fr.n;
    const int nt = (n + kTile - 1) / kTile;
    const int t = blockIdx.x;
    if (t >= nt * (nt + 1) / 2) return;
    int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);   // FP32 estimate, fixed below
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
    // per tile row / column: its dof, the two children's positions, the scale
    __shared__ int s_fd[2][kTile], s_iv[2][2][kTile];
    __shared__ double s_ds[2][kTile];
    for (int x = threadIdx.x; x < 2 * kTile; x += blockDim.x) {
        const int side = x / kTile, o = x % kTile;
        const int g = (side == 0 ? ti : tj) * kTile + o;
        int dd = 0, a0 = -1, a1 = -1;
        double sc = 0.0;
        if (g < n) { dd = fd[g]; a0 = inv0[g]; a1 = inv1[g]; sc = dscale[dd]; }
        s_fd[side][o] = dd; s_iv[side][0][o] = a0; s_iv[side][1][o] = a1; s_ds[side][o] = sc;
    }
    __syncthreads();
    // kBatch entries per thread at a time: all their child loads are issued
    // before any is used
    constexpr int kBatch = 8;
    for (int e0 = threadIdx.x; e0 < kTile * kTile; e0 += kBatch * blockDim.x) {
        double x[2][kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            const int rl = e / kTile, ql = e % kTile;
            const int r = ti * kTile + rl, q = tj * kTile + ql;
            const bool in = e < kTile * kTile && r < n && q <= r;
#pragma unroll
            for (int ci = 0; ci < 2; ++ci) {
                const int ir = in ? s_iv[0][ci][rl] : -1, iq = in ? s_iv[1][ci][ql] : -1;
                double v = 0.0;
                if (ir >= 0 && iq >= 0) {
                    const long long a = leaf[ci] ? (long long)ir * ld[ci] + iq
                                                 : (long long)(off[ci] + max(ir, iq)) * ld[ci] + off[ci] + min(ir, iq);
                    v = src[ci][a];
                }
                x[ci][u] = v;
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            const int rl = e / kTile, ql = e % kTile;
            const int r = ti * kTile + rl, q = tj * kTile + ql;
            if (e >= kTile * kTile || r >= n || q > r) continue;
            double v = 0.0;
#pragma unroll
            for (int ci = 0; ci < 2; ++ci)
                v += leaf[ci] ? dof_sign(s_fd[0][rl], NV) * x[ci][u] * s_ds[0][rl] * s_ds[1][ql] : x[ci][u];
            if (r == fr.pin_row && q == fr.pin_row) v -= 1.0;
            Fm[(long long)r * n + q] = v;
        }
    }
    if (t == 0 && fr.ne > 0) {              // first panel's diagonal block (inside tile (0, 0))
        __shared__ double work[kDiagWork];
        factor_diag_block(Fm, n, 0, min(kPanel, fr.ne), P + (long long)fr.p_off * kPanel * kPanel, status, work);
    }
}

constexpr int kPanelRows = 4;           // warp passes per panel-kernel CTA (one per warp)

// Tensor-core emulation of the FP64 trailing update (Ozaki-type splitting
// with exact integer arithmetic).  For each panel row x (of L21 D for the left
// operand, of L21 for the right one) let E be the smallest power of two with
// |x_k| < 2^E for every k of the row; |x_k| 2^{-E} is cut into S = 8 slices of
// 7 bits, x_k = 2^E sum_t s_t 2^{-7(t+1)} + r with integer |s_t| <= 127 and
// |r| < 2^{E-56} (sign carried by every slice), extracted from the bits of
// the double with integer operations.  Then
//   sum_k x_ik y_jk = 2^{E_i + F_j} sum_d P_d 2^{-7(d+2)},
//   P_d = sum_{t+u=d} sum_k s_t(x_ik) s_u(y_jk),   d = 0 .. S-1
// (terms with t + u >= S are below the FP64 rounding of the result).  Each
// P_d is a BF16 MMA with FP32 accumulation whose every partial sum is an
// integer below 2^22, hence exact; the P_d are combined exactly in 64-bit
// integers and converted to FP64 once.  An update then costs about five FP64
// operations per entry instead of one FMA per panel column.
constexpr int kOzS = 8;                     // slices per operand
constexpr int kOzRowWords = 2 * kOzS * kPanel / 2;   // u32 words per slice row (2 operands x 8 slices x 32 bf16)

__device__ __forceinline__ bool oz_step(const FrontInfo& fr, int m, int nbk) {
    return fr.s_off >= 0 && m >= kOzMinM && nbk >= kOzMinK;
}

// Maximum over the aligned segment of W lanes (W a power of two) holding this lane.
__device__ __forceinline__ unsigned long long seg_max_u64(unsigned long long v, int W) {
    for (int o = W >> 1; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Slices of one panel row held by a segment of W lanes (lane j of the segment
// holds column j; columns W .. 31 are zero) into `dst` (kOzS x 32 bf16) and
// its exponent E into *exp_out.  Integer operations only.
__device__ __forceinline__ void oz_slice_row(double x, int j, int W, bool store, __nv_bfloat16* dst, int* exp_out) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned long long mag = bits & 0x7FFFFFFFFFFFFFFFull;          // orders like |x|
    const unsigned long long mx = seg_max_u64(mag, W);
    const int E = mx == 0 ? 0 : (int)(mx >> 52) - 1023 + 1;                // max |x| < 2^E
    const int ex = (int)(mag >> 52);
    unsigned long long Fx = 0;                                             // floor(|x| 2^{56-E})
    if (ex != 0) {
        const unsigned long long mant = (mag & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = ex - 1023 + 4 - E;                                  // <= 3
        Fx = sh >= 0 ? (mant << sh) : (-sh < 64 ? (mant >> -sh) : 0ull);
    }
    const bool neg = (bits >> 63) != 0;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
    if (!store) return;                                                    // after the segment reduction
#pragma unroll
    for (int t = 0; t < kOzS; ++t) {
        const int v = (int)((Fx >> (49 - 7 * t)) & 127ull);
        dst[t * kPanel + j] = __float2bfloat16_rn((float)(neg ? -v : v));
        for (int c = j + W; c < kPanel; c += W) dst[t * kPanel + c] = zero;
    }
    if (j == 0) *exp_out = E;
}

// Slices of one panel row held as pairs: lane p of a 16-lane segment holds
// columns p and 31 - p (values x1, x2).  Same slices and exponent as
// oz_slice_row over the full row.
__device__ __forceinline__ unsigned long long oz_fixed(unsigned long long mag, int E) {   // floor(|x| 2^{56-E})
    const int ex = (int)(mag >> 52);
    if (ex == 0) return 0ull;
    const unsigned long long mant = (mag & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = ex - 1023 + 4 - E;                                      // <= 3
    return sh >= 0 ? (mant << sh) : (-sh < 64 ? (mant >> -sh) : 0ull);
}
__device__ __forceinline__ void oz_slice_pair(double x1, double x2, int p, bool store, __nv_bfloat16* dst,
                                              int* exp_out) {
    const unsigned long long b1 = (unsigned long long)__double_as_longlong(x1);
    const unsigned long long b2 = (unsigned long long)__double_as_longlong(x2);
    const unsigned long long m1 = b1 & 0x7FFFFFFFFFFFFFFFull, m2 = b2 & 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long mx = seg_max_u64(m1 > m2 ? m1 : m2, 16);
    const int E = mx == 0 ? 0 : (int)(mx >> 52) - 1023 + 1;
    const unsigned long long F1 = oz_fixed(m1, E), F2 = oz_fixed(m2, E);
    if (!store) return;                                                    // after the segment reduction
    const bool n1 = (b1 >> 63) != 0, n2 = (b2 >> 63) != 0;
#pragma unroll
    for (int t = 0; t < kOzS; ++t) {
        const int v1 = (int)((F1 >> (49 - 7 * t)) & 127ull), v2 = (int)((F2 >> (49 - 7 * t)) & 127ull);
        dst[t * kPanel + p] = __float2bfloat16_rn((float)(n1 ? -v1 : v1));
        dst[t * kPanel + kPanel - 1 - p] = __float2bfloat16_rn((float)(n2 ? -v2 : v2));
    }
    if (p == 0) *exp_out = E;
}

// Panel step of the blocked LDL^T: the rows below the (already factored)
// diagonal block, l = a L11^{-T} D^{-1}, i.e. l_j = sum_{k <= j} a_k V[j][k] / d_j
// with V = L11^{-1}.  Panels wider than 16 columns: a warp holds two rows,
// lane p of each half computes columns p and 31 - p (p + 1 and 32 - p terms of
// the triangular product, 33 FMAs in two chains instead of 32 per column), 8
// rows per CTA.  Narrower panels: a warp holds 32 / W rows at once, W = the
// panel width rounded up to a power of two (one lane per column), so narrow
// panels do not waste FP64 issue slots; kPanelRows x 32 / W rows per CTA.
__global__ void __launch_bounds__(128)
k_ldl_panel(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids, int k0, double* __restrict__ F,
            const double* __restrict__ P, __nv_bfloat16* __restrict__ oz, int* __restrict__ oz_exp) {
    pdl_begin();
    const FrontInfo fr = fronts[ids[blockIdx.y]];
    if (k0 >= fr.ne) return;
    const int n = fr.n;
    const int nbk = min(kPanel, fr.ne - k0);
    const int k1 = k0 + nbk;
    const int W = nbk <= 1 ? 1 : 1 << (32 - __clz(nbk - 1));
    const int R = kPanel / W;                                   // rows per warp pass
    const int rows = W == kPanel ? 2 * kPanelRows : kPanelRows * R;   // rows of this CTA
    const int r0 = k1 + blockIdx.x * rows;
    if (r0 >= n) return;
    const int r_end = min(n, r0 + rows);
    double* A = F + fr.f_off;
    __shared__ double Vs[kPanel][kPanel + 1];
    __shared__ double Dinv[kPanel], Dd[kPanel];
    const double* V = P + (long long)(fr.p_off + k0 / kPanel) * kPanel * kPanel;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < kPanel * kPanel; e += blockDim.x) Vs[e >> 5][e & 31] = V[e];
    if (threadIdx.x < kPanel) {
        const double d = threadIdx.x < nbk ? A[(long long)(k0 + threadIdx.x) * n + k0 + threadIdx.x] : 0.0;
        Dd[threadIdx.x] = d;
        Dinv[threadIdx.x] = threadIdx.x < nbk ? rcp64(d) : 0.0;
    }
    __syncthreads();
    const bool oz_on = oz_step(fr, n - k1, nbk);
    if (W == kPanel) {
        __shared__ double As[kPanelRows][2][kPanel];
        const int h = lane >> 4, p = lane & 15, p2 = kPanel - 1 - p;
        const int r = r0 + 2 * w + h;
        const bool live = r < r_end;
        double* row = A + (long long)min(r, r_end - 1) * n + k0;
        double* as = As[w][h];
        as[p] = (live && p < nbk) ? row[p] : 0.0;
        as[p2] = (live && p2 < nbk) ? row[p2] : 0.0;
        __syncwarp();
        // chain A: terms q = 0 .. 16 (column p while q <= p, then column p2);
        // chain B: q = 17 .. 32, all of column p2 (k = q - p - 1)
        double x1 = 0.0, x2 = 0.0, y2 = 0.0;
#pragma unroll
        for (int q = 0; q < 17; ++q) {
            const bool f = q <= p;
            const int k = f ? q : q - p - 1;
            const double v = fma(as[k], Vs[f ? p : p2][k], f ? x1 : x2);
            if (f) x1 = v; else x2 = v;
            if (q < 16) y2 = fma(as[q + 16 - p], Vs[p2][q + 16 - p], y2);
        }
        const double l1 = x1 * Dinv[p], l2 = (x2 + y2) * Dinv[p2];
        if (live && p < nbk) row[p] = l1;
        if (live && p2 < nbk) row[p2] = l2;
        if (oz_on) {                                              // all lanes: segment reductions inside
            const long long sr = (long long)fr.s_off + min(r, r_end - 1);
            oz_slice_pair(l1 * Dd[p], l2 * Dd[p2], p, live, oz + sr * (2 * kOzS * kPanel), oz_exp + 2 * sr);
            oz_slice_pair(l1, l2, p, live, oz + sr * (2 * kOzS * kPanel) + kOzS * kPanel, oz_exp + 2 * sr + 1);
        }
        return;
    }
    const int rs = lane / W, j = lane % W;
    for (int base = r0 + w * R; base < r_end; base += 4 * R) {
        const int r = base + rs;
        const bool live = r < r_end && j < nbk;
        double* row = A + (long long)r * n + k0;
        const double a = live ? row[j] : 0.0;
        double acc0 = 0.0, acc1 = 0.0;                            // two chains of FP64 FMAs
        int k = 0;
        for (; k + 1 < nbk; k += 2) {
            const double ak0 = __shfl_sync(0xffffffffu, a, rs * W + k);
            const double ak1 = __shfl_sync(0xffffffffu, a, rs * W + k + 1);
            acc0 = fma(ak0, Vs[j][k], acc0);                     // V[j][k] = 0 for k > j
            acc1 = fma(ak1, Vs[j][k + 1], acc1);
        }
        if (k < nbk) acc0 = fma(__shfl_sync(0xffffffffu, a, rs * W + k), Vs[j][k], acc0);
        const double l = live ? (acc0 + acc1) * Dinv[j] : 0.0;
        if (live) row[j] = l;
        if (oz_on) {                                              // all lanes: segment reductions inside
            const long long sr = (long long)fr.s_off + min(r, r_end - 1);
            oz_slice_row(l * Dd[j], j, W, r < r_end, oz + sr * (2 * kOzS * kPanel), oz_exp + 2 * sr);
            oz_slice_row(l, j, W, r < r_end, oz + sr * (2 * kOzS * kPanel) + kOzS * kPanel, oz_exp + 2 * sr + 1);
        }
    }
}

// BF16 m16n8k16 tensor-core MMA with FP32 accumulation (the emulated update
// feeds it small integers, for which it is exact).
__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], const uint32_t b[2]) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// The 128-bit integer v, times 2^e, rounded to the nearest FP64 value with
// integer operations only (ties away from zero; results below the normal
// range become 0).
__device__ __forceinline__ double i128_scaled(__int128 v, int e) {
    if (v == 0) return 0.0;
    const unsigned long long sign = v < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned __int128 m = v < 0 ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const unsigned long long mh = (unsigned long long)(m >> 64), ml = (unsigned long long)m;
    const int top = mh ? 127 - __clzll((long long)mh) : 63 - __clzll((long long)ml);   // m in [2^top, 2^(top+1))
    unsigned long long mant;                                   // top 53 bits, rounded
    int ex = top + e;
    if (top <= 52) {
        mant = ml << (52 - top);
    } else {
        const int sh = top - 52;
        const unsigned __int128 q = m >> sh;
        const bool up = (m >> (sh - 1)) & 1;                   // first dropped bit
        mant = (unsigned long long)q + (up ? 1ull : 0ull);
        if (mant >> 53) { mant >>= 1; ++ex; }                  // rounding carried into a new bit
    }
    const int be = ex + 1023;
    if (be <= 0) return 0.0;
    return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (mant & 0x000FFFFFFFFFFFFFull)));
}

// Exact integer value (|v| < 2^22) of an FP32 holding one: add 1.5 2^23 and
// read the significand (FP32 add and integer subtract, no conversion).
__device__ __forceinline__ int f32_int(float v) { return __float_as_int(v + 12582912.0f) - 0x4B400000; }

// Trailing update of the blocked LDL^T: F22 -= L21 D L21^T on 32 x 32 tiles
// of the lower triangle (small tiles spread one front's update over many
// SMs); blockIdx.x enumerates the (ti >= tj) tile pairs.  Large steps take
// the tensor-core emulation above, the others plain FP64 FMAs.  The CTA of
// tile (0, 0), which holds the next panel's diagonal block, factors that
// block afterwards.
constexpr int kOzLd = kOzRowWords / 2 + 4;  // u32 words per staged operand row (one operand, padded)
__global__ void __launch_bounds__(kThreads)
k_ldl_update(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids, int k0, double* __restrict__ F,
             double* __restrict__ P, int* __restrict__ status, const __nv_bfloat16* __restrict__ oz,
             const int* __restrict__ oz_exp) {
    pdl_begin();
    const FrontInfo fr = fronts[ids[blockIdx.y]];
    if (k0 >= fr.ne) return;
    const int n = fr.n;
    const int nbk = min(kPanel, fr.ne - k0);
    const int k1 = k0 + nbk;
    const int m = n - k1;
    if (m <= 0) return;
    const int nt = (m + kPanel - 1) / kPanel;
    const int T = nt * (nt + 1) / 2;
    const int t = blockIdx.x;
    if (t >= T) return;
    int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);   // FP32 estimate, fixed below
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    const int tj = t - ti * (ti + 1) / 2;
    double* A = F + fr.f_off;
    __shared__ __align__(16) uint32_t sbuf[2 * kPanel * kOzLd];             // 33.8 KB, reused below
    const int i0 = k1 + ti * kPanel, j0 = k1 + tj * kPanel;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (oz_step(fr, m, nbk)) {
        uint32_t* Sa = sbuf;                                               // rows i: slices of L21 D
        uint32_t* Sb = sbuf + kPanel * kOzLd;                              // rows j: slices of L21
        __shared__ int ez[2 * kPanel];                                     // row exponents E_i, F_j
        if (threadIdx.x < 2 * kPanel) {
            const int op = threadIdx.x / kPanel, rr = threadIdx.x % kPanel;
            const int gr = (op == 0 ? i0 : j0) + rr;
            ez[threadIdx.x] = gr < n ? oz_exp[2 * ((long long)fr.s_off + gr) + op] : 0;
        }
        const uint4* src = reinterpret_cast<const uint4*>(oz);
        for (int e = threadIdx.x; e < 2 * kPanel * (kOzLd - 4) / 4; e += blockDim.x) {
            const int op = e / (kPanel * (kOzLd - 4) / 4);
            const int rem = e % (kPanel * (kOzLd - 4) / 4);
            const int rr = rem / ((kOzLd - 4) / 4), q = rem % ((kOzLd - 4) / 4);
            const int gr = (op == 0 ? i0 : j0) + rr;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gr < n) v = src[((long long)fr.s_off + gr) * (kOzRowWords / 4) + op * ((kOzLd - 4) / 4) + q];
            reinterpret_cast<uint4*>((op == 0 ? Sa : Sb) + rr * kOzLd)[q] = v;
        }
        __syncthreads();
        const int g = lane >> 2, tg = lane & 3;
        const int mr = (w >> 2) * 16, nc = (w & 3) * 8;                   // this warp's 16 x 8 output block
        float acc[kOzS][4];
#pragma unroll
        for (int d = 0; d < kOzS; ++d)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[d][q] = 0.f;
        // P_d accumulates every slice pair (ts, us) with ts + us = d; consecutive
        // MMAs go to different accumulators
#pragma unroll
        for (int ts = 0; ts < kOzS; ++ts) {
            uint32_t af[2][4];
#pragma unroll
            for (int kc = 0; kc < 2; ++kc) {
                const int wa = ts * (kPanel / 2) + kc * 8 + tg;
                af[kc][0] = Sa[(mr + g) * kOzLd + wa];
                af[kc][1] = Sa[(mr + g + 8) * kOzLd + wa];
                af[kc][2] = Sa[(mr + g) * kOzLd + wa + 4];
                af[kc][3] = Sa[(mr + g + 8) * kOzLd + wa + 4];
            }
#pragma unroll
            for (int us = 0; us < kOzS - ts; ++us) {
#pragma unroll
                for (int kc = 0; kc < 2; ++kc) {
                    const int wb = us * (kPanel / 2) + kc * 8 + tg;
                    const uint32_t bf[2] = {Sb[(nc + g) * kOzLd + wb], Sb[(nc + g) * kOzLd + wb + 4]};
                    mma_bf16(acc[ts + us], af[kc], bf);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // S = sum_d P_d 2^{7(7-d)} exactly (|S| < 2^72), then one rounding to FP64
            __int128 sum = 0;
#pragma unroll
            for (int d = 0; d < kOzS; ++d) sum += (__int128)f32_int(acc[d][q]) << (7 * (7 - d));
            const int gi = i0 + mr + g + (q >> 1) * 8;
            const int gj = j0 + nc + 2 * tg + (q & 1);
            if (gi < n && gj <= gi) {
                const int e = ez[mr + g + (q >> 1) * 8] + ez[kPanel + nc + 2 * tg + (q & 1)];
                double* c = A + (long long)gi * n + gj;
                *c -= i128_scaled(sum, e - 63);
            }
        }
    } else {
        double (*Li)[kPanel + 1] = reinterpret_cast<double (*)[kPanel + 1]>(sbuf);
        double (*Lj)[kPanel + 1] = Li + kPanel;
        __shared__ double Dk[kPanel];
        if (threadIdx.x < kPanel) Dk[threadIdx.x] = threadIdx.x < nbk ? A[(long long)(k0 + threadIdx.x) * n + k0 + threadIdx.x] : 0.0;
        __syncthreads();
        for (int a = w; a < kPanel; a += kThreads / 32) {
            const int gi = i0 + a, gj = j0 + a;
            Li[a][lane] = (gi < n && lane < nbk) ? A[(long long)gi * n + k0 + lane] * Dk[lane] : 0.0;
            Lj[a][lane] = (gj < n && lane < nbk) ? A[(long long)gj * n + k0 + lane] : 0.0;
        }
        __syncthreads();
        const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;       // 16 x 16 threads, 2 x 2 outputs each
        double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
#pragma unroll 4
        for (int k = 0; k < nbk; ++k) {
            const double a0 = Li[ty][k], a1 = Li[ty + 16][k];
            const double b0 = Lj[tx][k], b1 = Lj[tx + 16][k];
            acc[0][0] = fma(a0, b0, acc[0][0]); acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]); acc[1][1] = fma(a1, b1, acc[1][1]);
        }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int gi = i0 + ty + 16 * p;
            if (gi >= n) continue;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int gj = j0 + tx + 16 * q;
                if (gj <= gi) A[(long long)gi * n + gj] -= acc[p][q];
            }
        }
    }
    if (t == 0 && k1 < fr.ne) {
        const int nb2 = min(kPanel, fr.ne - k1);
        __syncthreads();                                                   // shared buffer free for reuse
        factor_diag_block(A, n, k1, nb2, P + (long long)(fr.p_off + k1 / kPanel) * kPanel * kPanel, status,
                          reinterpret_cast<double*>(sbuf));
    }
}

// Forward substitution, eliminated part of one front (one CTA per front):
// r = children's reduced rhs + the scaled, J-signed global rhs of its E dofs,
// then L_EE y = r_E panel by panel (y_p = V_p r_p, rows below updated).  y_E
// and the B part of r (not yet reduced by y_E) go to frhs.
__global__ void __launch_bounds__(kThreads)
k_front_forward(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids,
                const int* __restrict__ maps, const int* __restrict__ dofs,
                const double* __restrict__ F, const double* __restrict__ P, const double* __restrict__ bglob,
                const double* __restrict__ dscale, int NV, double* __restrict__ frhs) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* r = reinterpret_cast<double*>(smem_raw);
    const FrontInfo fr = fronts[ids[blockIdx.x]];
    const int n = fr.n, ne = fr.ne;
    const double* A = F + fr.f_off;
    const int* fd = dofs + fr.e_dof_off;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
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
    __shared__ double Vs[kPanel][kPanel + 1];
    for (int k0 = 0; k0 < ne; k0 += kPanel) {
        const int nbk = min(kPanel, ne - k0), k1 = k0 + nbk;
        const double* V = P + (long long)(fr.p_off + k0 / kPanel) * kPanel * kPanel;
        for (int e = threadIdx.x; e < kPanel * kPanel; e += blockDim.x) Vs[e >> 5][e & 31] = V[e];
        __syncthreads();
        if (w == 0) {
            const double rk = lane < nbk ? r[k0 + lane] : 0.0;
            double y = 0.0;
#pragma unroll
            for (int k = 0; k < kPanel; ++k) y = fma(Vs[lane][k], __shfl_sync(0xffffffffu, rk, k), y);
            if (lane < nbk) r[k0 + lane] = y;
        }
        __syncthreads();
        for (int i = k1 + threadIdx.x; i < ne; i += blockDim.x) {       // one thread per row: 32 loads in flight
            const double* row = A + (long long)i * n + k0;
            double v = 0.0;
            if (nbk == kPanel) {
#pragma unroll
                for (int k = 0; k < kPanel; ++k) v = fma(row[k], r[k0 + k], v);
            } else {
                for (int k = 0; k < nbk; ++k) v = fma(row[k], r[k0 + k], v);
            }
            r[i] -= v;
        }
        __syncthreads();
    }
    double* out = frhs + fr.r_off;
    for (int q = threadIdx.x; q < n; q += blockDim.x) out[q] = r[q];
}

// Forward substitution, boundary rows: r_B -= L_BE y_E, one warp per row,
// kSolveRows rows per CTA, many CTAs per front.
constexpr int kSolveRows = 8;
__global__ void __launch_bounds__(kThreads)
k_front_forward_b(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids, const double* __restrict__ F,
                  double* __restrict__ frhs) {
    pdl_begin();
    const FrontInfo fr = fronts[ids[blockIdx.y]];
    const int n = fr.n, ne = fr.ne;
    const int i = ne + blockIdx.x * kSolveRows + (threadIdx.x >> 5);
    if (i >= n) return;
    const int lane = threadIdx.x & 31;
    const double* row = F + fr.f_off + (long long)i * n;
    double* rr = frhs + fr.r_off;
    double v = 0.0;
    for (int k = lane; k < ne; k += 32) v = fma(row[k], rr[k], v);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) rr[i] -= v;
}

// Backward substitution, boundary columns: w_E = D^{-1} y_E - L_BE^T x_B, with
// x_B (scaled) from the ancestors.  32 columns x 8 row groups per CTA, eight
// partial sums per thread; the boundary rows are cut into gridDim.z chunks
// (one CTA each, its x_B chunk gathered into shared memory).  With several
// chunks each CTA stores its column sums, and the CTA that completes a column
// block (counter wrapping back to 0, so the counters are ready for the next
// level) adds them in chunk order: the result does not depend on timing.
__global__ void __launch_bounds__(kThreads)
k_front_backward_b(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids, const int* __restrict__ dofs,
                   const double* __restrict__ F, const double* __restrict__ xs, double* __restrict__ frhs,
                   double* __restrict__ bpart, unsigned* __restrict__ bcnt) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* xb = reinterpret_cast<double*>(smem_raw);
    const FrontInfo fr = fronts[ids[blockIdx.y]];
    const int n = fr.n, ne = fr.ne, nb = n - ne;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    if (blockIdx.x * 32 >= ne) return;
    const int Z = gridDim.z, z = blockIdx.z;
    const int chunk = (nb + Z - 1) / Z;
    const int q0 = min(nb, z * chunk), q1 = min(nb, q0 + chunk);
    const double* A = F + fr.f_off;
    const int* fd = dofs + fr.e_dof_off;
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) xb[q - q0] = xs[fd[ne + q]];
    __shared__ double part[kThreads / 32][32];
    __shared__ unsigned last;
    __syncthreads();
    constexpr int G = kThreads / 32;
    double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};      // eight loads in flight per thread
    if (i < ne) {
        const double* col = A + (long long)ne * n + i;
        int q = q0 + g;
        for (; q + 7 * G < q1; q += 8 * G) {
            double a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = col[(long long)(q + u * G) * n];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = fma(a[u], xb[q - q0 + u * G], v[u]);
        }
        for (; q < q1; q += G) v[0] = fma(col[(long long)q * n], xb[q - q0], v[0]);
    }
    part[g][lane] = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    __syncthreads();
    double s = 0.0;
    if (g == 0) {
#pragma unroll
        for (int q = 0; q < G; ++q) s += part[q][lane];
    }
    double* zr = frhs + fr.r_off;
    if (Z == 1) {
        if (g == 0 && i < ne) zr[i] = zr[i] / A[(long long)i * n + i] - s;
        return;
    }
    const long long slot = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    if (g == 0) bpart[(slot * Z + z) * 32 + lane] = s;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicInc(&bcnt[slot], (unsigned)(Z - 1)) == (unsigned)(Z - 1);
    __syncthreads();
    if (last && g == 0 && i < ne) {
        __threadfence();
        double t = 0.0;
        for (int zz = 0; zz < Z; ++zz) t += __ldcg(&bpart[(slot * Z + zz) * 32 + lane]);
        zr[i] = zr[i] / A[(long long)i * n + i] - t;
    }
}

// Backward substitution, eliminated part (one CTA per front): L_EE^T x_E = w_E
// panel by panel from the last (x_p = V_p^T w_p, earlier entries updated).
__global__ void __launch_bounds__(kThreads)
k_front_backward(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids,
                 const int* __restrict__ dofs, const double* __restrict__ F, const double* __restrict__ P,
                 const double* __restrict__ frhs, double* __restrict__ xs) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* w = reinterpret_cast<double*>(smem_raw);
    const FrontInfo fr = fronts[ids[blockIdx.x]];
    const int n = fr.n, ne = fr.ne;
    const double* A = F + fr.f_off;
    const int* fd = dofs + fr.e_dof_off;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < ne; i += blockDim.x) w[i] = frhs[fr.r_off + i];
    __syncthreads();
    __shared__ double Vs[kPanel][kPanel + 1];
    const int nblk = (ne + kPanel - 1) / kPanel;
    for (int bk = nblk - 1; bk >= 0; --bk) {
        const int k0 = bk * kPanel, nbk = min(kPanel, ne - k0);
        const double* V = P + (long long)(fr.p_off + bk) * kPanel * kPanel;
        for (int e = threadIdx.x; e < kPanel * kPanel; e += blockDim.x) Vs[e >> 5][e & 31] = V[e];
        __syncthreads();
        if (wp == 0) {
            const double wk = lane < nbk ? w[k0 + lane] : 0.0;
            double x = 0.0;
#pragma unroll
            for (int k = 0; k < kPanel; ++k) x = fma(Vs[k][lane], __shfl_sync(0xffffffffu, wk, k), x);
            if (lane < nbk) w[k0 + lane] = x;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < k0; i += blockDim.x) {            // coalesced over i
            double acc = w[i];
            if (nbk == kPanel) {
#pragma unroll
                for (int k = 0; k < kPanel; ++k) acc = fma(-A[(long long)(k0 + k) * n + i], w[k0 + k], acc);
            } else {
                for (int k = 0; k < nbk; ++k) acc = fma(-A[(long long)(k0 + k) * n + i], w[k0 + k], acc);
            }
            w[i] = acc;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < ne; i += blockDim.x) xs[fd[i]] = w[i];
}

// ---------------------------------------------------------------------------
// Cluster variants of the two eliminated-part substitutions for large fronts:
// kSolveCl CTAs (one thread-block cluster) share a front.  Panel p belongs to
// CTA p mod kSolveCl, which keeps the rows (forward) or entries (backward) of
// its panels.  Per panel the owner solves the 32 x 32 diagonal system in one
// warp, writes the result into every CTA's shared memory (distributed shared
// memory), and a cluster barrier releases it; every CTA then applies it to its
// own later (forward) or earlier (backward) panels.  The FP64 updates, which
// bind a single SM, are spread over the cluster; the only waits are the
// hardware cluster barrier.
// ---------------------------------------------------------------------------
constexpr int kSolveCl = 8;
constexpr int kSolveClMinNe = 4 * kPanel;    // fronts with fewer E dofs keep one CTA
constexpr size_t kClSmemMax = 180 * 1024;    // dynamic shared memory cap of the cluster kernels

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// store v at the same shared-memory offset as `local` in CTA `rank` of the cluster
__device__ __forceinline__ void st_cluster(double* local, unsigned rank, double v) {
    unsigned la = (unsigned)__cvta_generic_to_shared(local), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
    asm volatile("st.shared::cluster.f64 [%0], %1;" :: "r"(ra), "d"(v) : "memory");
}

__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared memory of the cluster substitutions: the front's vector (n doubles,
// padded to 16 bytes), then the inverse diagonal blocks of this CTA's panels.
__host__ __device__ inline size_t cl_own_panels(int ne) { return ((ne + kPanel - 1) / kPanel + kSolveCl - 1) / kSolveCl; }
__host__ __device__ inline size_t cl_vec_bytes(int n) { return ((size_t)n * sizeof(double) + 15) & ~size_t(15); }
__host__ __device__ inline size_t cl_smem_bytes(int n, int ne) {
    return cl_vec_bytes(n) + cl_own_panels(ne) * kPanel * (kPanel + 1) * sizeof(double);
}

// Copy this CTA's inverse diagonal blocks (panels q, q + kSolveCl, ...) into Vown.
__device__ __forceinline__ void cl_load_own_v(const double* __restrict__ P, const FrontInfo& fr, unsigned q, int np,
                                              double* Vown) {
    for (int j = 0; q + (unsigned)j * kSolveCl < (unsigned)np; ++j) {
        const double* V = P + (long long)(fr.p_off + q + j * kSolveCl) * kPanel * kPanel;
        double* D = Vown + (size_t)j * kPanel * (kPanel + 1);
        for (int e = threadIdx.x; e < kPanel * kPanel; e += blockDim.x) D[(e >> 5) * (kPanel + 1) + (e & 31)] = V[e];
    }
}

__global__ void __launch_bounds__(kThreads)
k_front_forward_cl(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids,
                   const int* __restrict__ maps, const int* __restrict__ dofs,
                   const double* __restrict__ F, const double* __restrict__ P, const double* __restrict__ bglob,
                   const double* __restrict__ dscale, int NV, double* __restrict__ frhs) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double ybuf[2][kPanel];
    const unsigned q = cluster_rank();
    const FrontInfo fr = fronts[ids[blockIdx.x / kSolveCl]];
    const int n = fr.n, ne = fr.ne;
    const int np = (ne + kPanel - 1) / kPanel;
    double* r = reinterpret_cast<double*>(smem_raw);
    double* Vown = reinterpret_cast<double*>(smem_raw + cl_vec_bytes(n));
    const double* A = F + fr.f_off;
    const int* fd = dofs + fr.e_dof_off;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    cl_load_own_v(P, fr, q, np, Vown);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v = 0.0;
        if (i < ne) { int d = fd[i]; v = dof_sign(d, NV) * dscale[d] * bglob[d]; }
        r[i] = v;
    }
    __syncthreads();
    for (int ci = 0; ci < 2; ++ci) {
        const int c = fr.child[ci];
        if (c < 0) continue;
        const FrontInfo cf = fronts[c];
        const int* mp = maps + fr.map_off[ci];
        for (int i = threadIdx.x; i < cf.nb; i += blockDim.x) r[mp[i]] += frhs[cf.r_off + cf.ne + i];
        __syncthreads();
    }
    cluster_sync_all();                                     // every CTA of the cluster is running
    for (int p = 0; p < np; ++p) {
        const int k0 = p * kPanel, nbk = min(kPanel, ne - k0);
        double* yb = ybuf[p & 1];
        if ((unsigned)(p % kSolveCl) == q && w == 0) {      // owner: y_p = V_p r_p, sent to the cluster
            const double* Vs = Vown + (size_t)(p / kSolveCl) * kPanel * (kPanel + 1);
            const double rk = lane < nbk ? r[k0 + lane] : 0.0;
            double y0 = 0.0, y1 = 0.0;
#pragma unroll
            for (int k = 0; k < kPanel; k += 2) {
                y0 = fma(Vs[lane * (kPanel + 1) + k], __shfl_sync(0xffffffffu, rk, k), y0);
                y1 = fma(Vs[lane * (kPanel + 1) + k + 1], __shfl_sync(0xffffffffu, rk, k + 1), y1);
            }
            const double y = y0 + y1;
            if (lane < nbk) r[k0 + lane] = y;
#pragma unroll
            for (unsigned t = 0; t < kSolveCl; ++t) st_cluster(&yb[lane], t, y);
        }
        cluster_arrive();
        // own rows of the later panels: r_i -= L[i][k0 .. k0 + nbk) y_p.  The
        // first own panel after p, then every kSolveCl-th; thread group
        // threadIdx.x / 32 takes every (kThreads / 32)-th of them, a lane per
        // row.  The first row's segment is read before the barrier completes.
        const int p1 = p + 1 + (int)((q + kSolveCl - (unsigned)((p + 1) % kSolveCl)) % kSolveCl);
        int pp = p1 + kSolveCl * (threadIdx.x / kPanel);
        int i = pp * kPanel + threadIdx.x % kPanel;
        double a[kPanel];
        const bool pre = pp < np && i < ne && nbk == kPanel;
        {
            const double* row = A + (pre ? (long long)i * n + k0 : 0);      // the front's first entries when idle
#pragma unroll
            for (int k = 0; k < kPanel; ++k) a[k] = pre ? row[k] : 0.0;
        }
        cluster_wait();                                     // y_p in every CTA
        if (pre) {
            double v0 = 0.0, v1 = 0.0;
#pragma unroll
            for (int k = 0; k < kPanel; k += 2) { v0 = fma(a[k], yb[k], v0); v1 = fma(a[k + 1], yb[k + 1], v1); }
            r[i] -= v0 + v1;
        }
        for (pp += pre ? kSolveCl * (kThreads / kPanel) : 0; pp < np; pp += kSolveCl * (kThreads / kPanel)) {
            i = pp * kPanel + threadIdx.x % kPanel;
            if (i >= ne) continue;
            const double* row = A + (long long)i * n + k0;
            double v0 = 0.0, v1 = 0.0;
            if (nbk == kPanel) {
#pragma unroll
                for (int k = 0; k < kPanel; k += 2) { v0 = fma(row[k], yb[k], v0); v1 = fma(row[k + 1], yb[k + 1], v1); }
            } else {
                for (int k = 0; k < nbk; ++k) v0 = fma(row[k], yb[k], v0);
            }
            r[i] -= v0 + v1;
        }
        __syncthreads();
    }
    double* out = frhs + fr.r_off;
    for (int p = q; p < np; p += kSolveCl)
        for (int i = p * kPanel + threadIdx.x; i < min(ne, p * kPanel + kPanel); i += blockDim.x) out[i] = r[i];
    if (q == 0)
        for (int i = ne + threadIdx.x; i < n; i += blockDim.x) out[i] = r[i];
    cluster_sync_all();                                     // no CTA leaves while others may write to it
}

__global__ void __launch_bounds__(kThreads)
k_front_backward_cl(const FrontInfo* __restrict__ fronts, const int* __restrict__ ids,
                    const int* __restrict__ dofs, const double* __restrict__ F, const double* __restrict__ P,
                    const double* __restrict__ frhs, double* __restrict__ xs) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int kChunk = 8;                               // own earlier panels per reduction round
    __shared__ double xbuf[2][kPanel];
    __shared__ double red[kChunk][kThreads / 32][kPanel];
    const unsigned q = cluster_rank();
    const FrontInfo fr = fronts[ids[blockIdx.x / kSolveCl]];
    const int n = fr.n, ne = fr.ne;
    const int np = (ne + kPanel - 1) / kPanel;
    double* wv = reinterpret_cast<double*>(smem_raw);
    double* Vown = reinterpret_cast<double*>(smem_raw + cl_vec_bytes(n));
    const double* A = F + fr.f_off;
    const int* fd = dofs + fr.e_dof_off;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    cl_load_own_v(P, fr, q, np, Vown);
    for (int i = threadIdx.x; i < ne; i += blockDim.x) wv[i] = frhs[fr.r_off + i];
    __syncthreads();
    cluster_sync_all();
    for (int p = np - 1; p >= 0; --p) {
        const int k0 = p * kPanel, nbk = min(kPanel, ne - k0);
        double* xb = xbuf[p & 1];
        if ((unsigned)(p % kSolveCl) == q && w == 0) {      // owner: x_p = V_p^T w_p, sent to the cluster
            const double* Vs = Vown + (size_t)(p / kSolveCl) * kPanel * (kPanel + 1);
            const double wk = lane < nbk ? wv[k0 + lane] : 0.0;
            double x0 = 0.0, x1 = 0.0;
#pragma unroll
            for (int k = 0; k < kPanel; k += 2) {
                x0 = fma(Vs[k * (kPanel + 1) + lane], __shfl_sync(0xffffffffu, wk, k), x0);
                x1 = fma(Vs[(k + 1) * (kPanel + 1) + lane], __shfl_sync(0xffffffffu, wk, k + 1), x1);
            }
            const double x = x0 + x1;
            if (lane < nbk) wv[k0 + lane] = x;
#pragma unroll
            for (unsigned t = 0; t < kSolveCl; ++t) st_cluster(&xb[lane], t, lane < nbk ? x : 0.0);
        }
        cluster_arrive();
        // own entries of the earlier panels pp = q, q + kSolveCl, ... < p:
        // w_i -= sum_k L[k0 + k][i] x_p[k], warp w taking k = w, w + 8, ...;
        // the first chunk's matrix entries are read before the barrier completes
        const int nown = p > (int)q ? (p - (int)q + kSolveCl - 1) / kSolveCl : 0;
        double a[kChunk][kPanel / (kThreads / 32)];
#pragma unroll
        for (int j = 0; j < kChunk; ++j)
#pragma unroll
            for (int u = 0; u < kPanel / (kThreads / 32); ++u) {
                const int k = w + u * (kThreads / 32);
                a[j][u] = (j < nown && k < nbk) ? A[(long long)(k0 + k) * n + (q + j * kSolveCl) * kPanel + lane] : 0.0;
            }
        cluster_wait();                                     // x_p in every CTA
        for (int j0 = 0; j0 < nown; j0 += kChunk) {
            if (j0 > 0) {
#pragma unroll
                for (int j = 0; j < kChunk; ++j)
#pragma unroll
                    for (int u = 0; u < kPanel / (kThreads / 32); ++u) {
                        const int k = w + u * (kThreads / 32);
                        a[j][u] = (j0 + j < nown && k < nbk)
                                      ? A[(long long)(k0 + k) * n + (q + (j0 + j) * kSolveCl) * kPanel + lane] : 0.0;
                    }
            }
#pragma unroll
            for (int j = 0; j < kChunk; ++j) {
                if (j0 + j >= nown) break;                  // FP64 instructions only for real panels
                double acc = 0.0;
#pragma unroll
                for (int u = 0; u < kPanel / (kThreads / 32); ++u) acc = fma(a[j][u], xb[w + u * (kThreads / 32)], acc);
                red[j][w][lane] = acc;
            }
            __syncthreads();
            if (w < kChunk && j0 + w < nown) {              // warp j sums entry lane of own panel j0 + j
                double sacc = 0.0;
#pragma unroll
                for (int g = 0; g < kThreads / 32; ++g) sacc += red[w][g][lane];
                wv[(q + (j0 + w) * kSolveCl) * kPanel + lane] -= sacc;
            }
            __syncthreads();
        }
    }
    for (int p = q; p < np; p += kSolveCl)
        for (int i = p * kPanel + threadIdx.x; i < min(ne, p * kPanel + kPanel); i += blockDim.x) xs[fd[i]] = wv[i];
    cluster_sync_all();
}

// r = b - (A^int - delta e0 e0^T) x   (CSR, FP64; delta = 1/d_0^2 when pinned)
__global__ void k_csr_residual(int nrows, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                               const double* __restrict__ val, const double* __restrict__ b,
                               const double* __restrict__ x, const double* __restrict__ dscale, int pin,
                               double* __restrict__ r) {
    pdl_begin();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    double acc = b[i];
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) acc -= val[q] * x[colidx[q]];
    if (pin && i == 0) acc += x[0] / (dscale[0] * dscale[0]);
    r[i] = acc;
}

__global__ void k_unscale(int n, const double* __restrict__ xs, const double* __restrict__ dscale,
                          double* __restrict__ x, int accumulate) {
    pdl_begin();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = xs[i] * dscale[i];
    x[i] = accumulate ? x[i] + v : v;
}

struct LevelPlan { int steps; std::vector<int> row_tiles, upd_tiles; int fwd_rows, bwd_cols, max_ne, max_nb; size_t cl_smem; };

LevelPlan plan_level(const Tables& t, int h) {
    LevelPlan p;
    int max_ne = 0, max_nb = 0;
    for (int id : t.levels[h]) { max_ne = std::max(max_ne, t.fronts[id].ne); max_nb = std::max(max_nb, t.fronts[id].nb); }
    p.steps = (max_ne + kPanel - 1) / kPanel;
    p.fwd_rows = std::max(1, (max_nb + kSolveRows - 1) / kSolveRows);
    p.bwd_cols = std::max(1, (max_ne + 31) / 32);
    p.max_ne = max_ne;
    p.max_nb = max_nb;
    p.cl_smem = 0;
    for (int id : t.levels[h]) p.cl_smem = std::max(p.cl_smem, cl_smem_bytes(t.fronts[id].n, t.fronts[id].ne));
    for (int s = 0; s < p.steps; ++s) {
        int k0 = s * kPanel, rt = 1, ut = 1;
        for (int id : t.levels[h]) {
            const FrontInfo& f = t.fronts[id];
            if (k0 >= f.ne) continue;
            int k1 = k0 + std::min(kPanel, f.ne - k0);
            int m = f.n - k1;
            rt = std::max(rt, (m + 2 * kPanelRows - 1) / (2 * kPanelRows));   // >= 8 rows per CTA
            int nt = (m + kPanel - 1) / kPanel;
            ut = std::max(ut, nt * (nt + 1) / 2);
        }
        p.row_tiles.push_back(rt);
        p.upd_tiles.push_back(ut);
    }
    return p;
}

}  // namespace

// Launch with programmatic stream serialization (see pdl_begin).
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

int launch_assemble_interface(const Tables& t, const DeviceTables& d, const Layout& L, char* ws, void* stream, Prof& P) {
    cudaStream_t st = (cudaStream_t)stream;
    const int nd = 2 * t.NV;
    if (nd == 0) return 0;
    double* dscale = (double*)(ws + L.dscale);
    MRCM_LAUNCH(P, "k_assemble_csr", st, launch_pdl(k_assemble_csr, dim3((nd + 127) / 128), dim3(128), 0, st, nd, d.rowptr, d.src_lo, d.src_hi, d.rhs_src_lo, d.rhs_src_hi,
                                                   d.colidx, (const double*)(ws + L.elem),
                                                   (const double*)(ws + L.elem_b), (double*)(ws + L.csr_val),
                                                   (double*)(ws + L.b_int), dscale, t.has_dirichlet ? 0 : 1));
    // numeric multifrontal factorisation, leaves to root
    double* F = (double*)(ws + L.fronts);
    double* Pv = (double*)(ws + L.panel);       // inverse diagonal blocks of the panels
    __nv_bfloat16* oz = (__nv_bfloat16*)(ws + L.oz);
    int* oz_exp = (int*)(ws + L.oz_exp);
    int* status = (int*)(ws + L.status);
    for (size_t h = 1; h < t.levels.size(); ++h) {
        int cnt = (int)t.levels[h].size();
        if (!cnt) continue;
        const int* ids = d.level_ids + d.level_off[h];
        int maxT = 1;
        for (int id : t.levels[h]) { int nt = (t.fronts[id].n + kTile - 1) / kTile; maxT = std::max(maxT, nt * (nt + 1) / 2); }
        dim3 ga(maxT, cnt);
        MRCM_LAUNCH(P, "k_front_assemble", st, launch_pdl(k_front_assemble, dim3(ga), dim3(kThreads), 0, st, d.fronts, ids, d.front_inv, d.front_dofs, d.subs,
                                                  (const double*)(ws + L.elem), dscale, t.NV, F, Pv, status));
        LevelPlan p = plan_level(t, (int)h);
        for (int s = 0; s < p.steps; ++s) {
            dim3 gp(p.row_tiles[s], cnt);
            MRCM_LAUNCH(P, "k_ldl_panel", st, launch_pdl(k_ldl_panel, dim3(gp), dim3(128), 0, st, d.fronts, ids, s * kPanel, F, Pv, oz, oz_exp));
            dim3 gu(p.upd_tiles[s], cnt);
            MRCM_LAUNCH(P, "k_ldl_update", st, launch_pdl(k_ldl_update, dim3(gu), dim3(kThreads), 0, st, d.fronts, ids, s * kPanel, F, Pv, status,
                                                                                   oz, oz_exp));
        }
    }
    return (int)cudaGetLastError();
}

// Launch `kern` as clusters of kSolveCl CTAs, one cluster per front of the level.
template <typename... Args>
static void launch_cluster(void (*kern)(Args...), int fronts, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(fronts * kSolveCl);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kSolveCl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

static void multifrontal_solve(const Tables& t, const DeviceTables& d, const Layout& L, char* ws,
                               const double* rhs, double* xs, cudaStream_t st, Prof& P) {
    double* F = (double*)(ws + L.fronts);
    const double* Pv = (const double*)(ws + L.panel);
    double* frhs = (double*)(ws + L.frhs);
    const double* dscale = (const double*)(ws + L.dscale);
    double* bpart = (double*)(ws + L.bpart);
    unsigned* bcnt = (unsigned*)(ws + L.bcnt);
    size_t sm = sizeof(double) * (size_t)std::max(t.max_front, 1);
    for (size_t h = 1; h < t.levels.size(); ++h) {
        int cnt = (int)t.levels[h].size();
        if (!cnt) continue;
        const int* ids = d.level_ids + d.level_off[h];
        const LevelPlan p = plan_level(t, (int)h);
        if (p.max_ne >= kSolveClMinNe && p.cl_smem <= kClSmemMax)
            MRCM_LAUNCH(P, "k_front_forward", st, launch_cluster(k_front_forward_cl, cnt, p.cl_smem, st, (const FrontInfo*)d.fronts, ids,
                                                                 (const int*)d.front_maps, (const int*)d.front_dofs, (const double*)F,
                                                                 Pv, rhs, dscale, (int)t.NV, frhs));
        else
            MRCM_LAUNCH(P, "k_front_forward", st, launch_pdl(k_front_forward, dim3(cnt), dim3(kThreads), sm, st, d.fronts, ids, d.front_maps,
                                                      d.front_dofs, F, Pv, rhs, dscale, t.NV, frhs));
        MRCM_LAUNCH(P, "k_front_forward_b", st, launch_pdl(k_front_forward_b, dim3(p.fwd_rows, cnt), dim3(kThreads), 0, st, d.fronts, ids, F, frhs));
    }
    for (size_t h = t.levels.size() - 1; h >= 1; --h) {
        int cnt = (int)t.levels[h].size();
        if (!cnt) continue;
        const int* ids = d.level_ids + d.level_off[h];
        const LevelPlan p = plan_level(t, (int)h);
        MRCM_LAUNCH(P, "k_front_backward_b", st, launch_pdl(k_front_backward_b, dim3(p.bwd_cols, cnt, bwd_split(p.max_nb)), dim3(kThreads), sm, st, 
                                                        d.fronts, ids, d.front_dofs, F, xs, frhs, bpart, bcnt));
        if (p.max_ne >= kSolveClMinNe && p.cl_smem <= kClSmemMax)
            MRCM_LAUNCH(P, "k_front_backward", st, launch_cluster(k_front_backward_cl, cnt, p.cl_smem, st, (const FrontInfo*)d.fronts, ids,
                                                                  (const int*)d.front_dofs, (const double*)F, Pv,
                                                                  (const double*)frhs, xs));
        else
            MRCM_LAUNCH(P, "k_front_backward", st, launch_pdl(k_front_backward, dim3(cnt), dim3(kThreads), sm, st, d.fronts, ids, d.front_dofs, F, Pv,
                                                       frhs, xs));
    }
}

int configure_interface(const Tables& t, DeviceTables& d) {
    // opt in to the dynamic shared memory each substitution kernel may take
    // (static + dynamic above 48 KB needs it)
    d.front_smem = sizeof(double) * (size_t)std::max(t.max_front, 1);
    cudaFuncSetAttribute(k_front_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.front_smem);
    cudaFuncSetAttribute(k_front_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.front_smem);
    cudaFuncSetAttribute(k_front_backward_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.front_smem);
    size_t cl = 0;
    for (const FrontInfo& f : t.fronts)
        if (f.ne >= kSolveClMinNe) cl = std::max(cl, cl_smem_bytes(f.n, f.ne));
    const int lim = (int)std::max<size_t>(std::min(cl, kClSmemMax), 1);
    cudaFuncSetAttribute(k_front_forward_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_front_backward_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
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
    {
        size_t parts, cnts;                     // counters of the split back substitution start at 0
        bwd_split_sizes(t.levels, t.fronts, &parts, &cnts);
        cudaMemsetAsync(ws + L.bcnt, 0, cnts * sizeof(unsigned), st);
    }
    multifrontal_solve(t, d, L, ws, b, xs, st, P);
    MRCM_LAUNCH(P, "k_unscale", st, launch_pdl(k_unscale, dim3((nd + 255) / 256), dim3(256), 0, st, nd, xs, dscale, X, 0));
    const int refine = t.cfg.interface_refine == 0 ? 1 : std::max(0, t.cfg.interface_refine);
    for (int it = 0; it < refine; ++it) {
        MRCM_LAUNCH(P, "k_csr_residual", st, launch_pdl(k_csr_residual, dim3((nd + 127) / 128), dim3(128), 0, st, nd, d.rowptr, d.colidx, (const double*)(ws + L.csr_val),
                                                       b, X, dscale, pin, r));
        multifrontal_solve(t, d, L, ws, r, xs, st, P);
        MRCM_LAUNCH(P, "k_unscale", st, launch_pdl(k_unscale, dim3((nd + 255) / 256), dim3(256), 0, st, nd, xs, dscale, X, 1));
    }
    return (int)cudaGetLastError();
}

}  // namespace mrcm
