// Reconstruction of the multiscale solution (Alg. MRCM second loop,
// ReconstructMscSolution, option 1 of the paper):
//   p^l = sum_k pi^p_k p(phi_k, 0) + pi^u_k p(0, phi_k) + pbar
// followed by face velocities: interior faces by Eq. two_point, Gamma faces
// by the Robin flux with the final data g = P_H - beta s U_H (each side keeps
// its own value), walls 0 (no-flow) or the Dirichlet half-cell flux.  The
// per-cell FP64 mass balance sum(out-fluxes) - f V is reduced to its maximum.
#include <cuda_runtime.h>

#include "mrcm_internal.h"

namespace mrcm {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxCells = 4096;

struct Geo2 {
    double h[3];
    double area[3];
    double inv_area[3];          // 1 / area: no FP64 divisions per face
    int n[3];
    int dir_lo, dir_hi;          // Dirichlet wall masks
    double glo[3], ghi[3];
};

__device__ __forceinline__ void lcoords(const SubInfo& s, int c, int lc[3]) {
    int sl = c / s.b;
    int r = c - sl * s.b;
    int v = r / s.su;
    lc[s.sa] = sl;
    lc[s.ua] = r - v * s.su;
    lc[s.va] = v;
}

__global__ void __launch_bounds__(kThreads)
k_reconstruct(const SubInfo* __restrict__ subs, const FaceInfo* __restrict__ faces,
              const int* __restrict__ Ilist, int NV, const double* __restrict__ Xmbf,
              const double* __restrict__ Xint, const double* __restrict__ coef,
              const double* __restrict__ face_tr, const double* __restrict__ face_beta,
              const double* __restrict__ K, const double* __restrict__ f, Geo2 geo, long long nct,
              double* __restrict__ p, double* __restrict__ u, double* __restrict__ psum,
              unsigned long long* __restrict__ mres_bits) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* pl = reinterpret_cast<double*>(smem_raw);        // N
    double* cvec = pl + kMaxCells;                          // m
    const SubInfo s = subs[blockIdx.x];
    const int N = s.N, m = s.m, nI = s.nI, b = s.b, su = s.su;
    const long long ncells = (long long)geo.n[0] * geo.n[1] * geo.n[2];
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double c;
        if (j < nI) c = Xint[Ilist[s.I_off + j]];
        else if (j < 2 * nI) c = Xint[NV + Ilist[s.I_off + j - nI]];
        else c = 1.0;
        cvec[j] = c;
    }
    __syncthreads();
    const double* Xs = Xmbf + s.x_off;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        // four independent FMA chains over the columns, added in a fixed order
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int j = 0;
        for (; j + 3 < m; j += 4) {
            a0 = fma(Xs[(long long)j * N + c], cvec[j], a0);
            a1 = fma(Xs[(long long)(j + 1) * N + c], cvec[j + 1], a1);
            a2 = fma(Xs[(long long)(j + 2) * N + c], cvec[j + 2], a2);
            a3 = fma(Xs[(long long)(j + 3) * N + c], cvec[j + 3], a3);
        }
        for (; j < m; ++j) a0 = fma(Xs[(long long)j * N + c], cvec[j], a0);
        pl[c] = (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
    const double* cu = coef + nct + s.cell_off;
    const double* cv = coef + 2 * nct + s.cell_off;
    const double* cs = coef + 3 * nct + s.cell_off;
    const long long strideg[3] = {1, geo.n[0], (long long)geo.n[0] * geo.n[1]};
    double psub = 0.0;
    // interior faces and walls
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        int lc[3];
        lcoords(s, c, lc);
        long long g = (s.o[0] + lc[0]) + geo.n[0] * ((long long)(s.o[1] + lc[1]) + (long long)geo.n[1] * (s.o[2] + lc[2]));
        psub += pl[c];
        p[g] = pl[c];
        const int r = c % b;
        const int uu = r % su;
        // local axis -> neighbour offset / transmissibility array
        for (int a = 0; a < 3; ++a) {
            int off;
            const double* tp;
            bool has_hi, has_lo;
            if (a == s.ua) { off = 1; tp = cu; has_hi = uu + 1 < su; has_lo = uu > 0; }
            else if (a == s.va) { off = su; tp = cv; has_hi = r + su < b; has_lo = r >= su; }
            else { off = b; tp = cs; has_hi = c + b < N; has_lo = c >= b; }
            const bool wall_lo = s.o[a] + lc[a] == 0;
            const bool wall_hi = s.o[a] + lc[a] == geo.n[a] - 1;
            double* ulo = u + (long long)(2 * a) * ncells;
            double* uhi = u + (long long)(2 * a + 1) * ncells;
            const double ka = K[(long long)a * ncells + g];
            if (has_hi) uhi[g] = tp[c] * (pl[c] - pl[c + off]) * geo.inv_area[a];
            else if (wall_hi) uhi[g] = ((geo.dir_hi >> a) & 1) ? -2.0 * ka * (geo.ghi[a] - pl[c]) / geo.h[a] : 0.0;
            if (has_lo) ulo[g] = tp[c - off] * (pl[c - off] - pl[c]) * geo.inv_area[a];
            else if (wall_lo) ulo[g] = ((geo.dir_lo >> a) & 1) ? -2.0 * ka * (pl[c] - geo.glo[a]) / geo.h[a] : 0.0;
            (void)strideg;
        }
    }
    // Robin faces
    for (int q = threadIdx.x; q < s.nface; q += blockDim.x) {
        FaceInfo fi = faces[s.face_off + q];
        int k = Ilist[s.I_off + fi.col];
        double be = face_beta[s.face_off + q];
        double gval = Xint[k] - be * fi.s * Xint[NV + k];
        double qo = face_tr[s.face_off + q] * (pl[fi.cell] - gval);
        int lc[3];
        lcoords(s, fi.cell, lc);
        long long g = (s.o[0] + lc[0]) + geo.n[0] * ((long long)(s.o[1] + lc[1]) + (long long)geo.n[1] * (s.o[2] + lc[2]));
        int a = fi.axis;
        if (fi.s > 0) u[(long long)(2 * a + 1) * ncells + g] = qo * geo.inv_area[a];
        else u[(long long)(2 * a) * ncells + g] = -qo * geo.inv_area[a];
    }
    __syncthreads();
    // mass balance of every cell of this subdomain
    const double vol = geo.h[0] * geo.h[1] * geo.h[2];
    double mx = 0.0;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        int lc[3];
        lcoords(s, c, lc);
        long long g = (s.o[0] + lc[0]) + geo.n[0] * ((long long)(s.o[1] + lc[1]) + (long long)geo.n[1] * (s.o[2] + lc[2]));
        double div = -f[g] * vol;
        for (int a = 0; a < 3; ++a)
            div += (u[(long long)(2 * a + 1) * ncells + g] - u[(long long)(2 * a) * ncells + g]) * geo.area[a];
        mx = (div == div) ? fmax(mx, fabs(div)) : __longlong_as_double(0x7ff0000000000000LL);
    }
    __shared__ double red[kThreads];
    __shared__ double redm[kThreads];
    red[threadIdx.x] = psub;
    redm[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[threadIdx.x] += red[threadIdx.x + w];
            redm[threadIdx.x] = fmax(redm[threadIdx.x], redm[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        psum[blockIdx.x] = red[0];
        atomicMax(mres_bits, (unsigned long long)__double_as_longlong(redm[0]));
    }
}

// Sum the per-subdomain partial sums in a fixed order and subtract the mean.
__global__ void k_mean(const double* __restrict__ psum, int nsub, long long ncells, double* __restrict__ mean) {
    __shared__ double red[kThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nsub; i += blockDim.x) acc += psum[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *mean = red[0] / (double)ncells;
}

__global__ void k_shift(double* __restrict__ p, long long n, const double* __restrict__ mean) {
    const double mu = *mean;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] -= mu;
}

__global__ void k_zero_u64(unsigned long long* x) { *x = 0ull; }

}  // namespace

int configure_reconstruct(const Tables& t) {
    cudaFuncSetAttribute(k_reconstruct, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(double) * ((size_t)kMaxCells + t.max_m)));
    return (int)cudaGetLastError();
}

int launch_reconstruct(const Tables& t, const DeviceTables& d, const Layout& L, char* ws,
                       const double* X, double* p, double* u, double* mres, const double* K,
                       const double* f, void* stream, Prof& P) {
    cudaStream_t st = (cudaStream_t)stream;
    const int nsub = (int)t.subs.size();
    const mrcm_config& c = t.cfg;
    Geo2 geo;
    geo.h[0] = c.hx; geo.h[1] = c.hy; geo.h[2] = c.hz;
    geo.area[0] = c.hy * c.hz; geo.area[1] = c.hx * c.hz; geo.area[2] = c.hx * c.hy;
    for (int a = 0; a < 3; ++a) geo.inv_area[a] = 1.0 / geo.area[a];
    geo.n[0] = c.nx; geo.n[1] = c.ny; geo.n[2] = c.nz;
    geo.dir_lo = geo.dir_hi = 0;
    for (int a = 0; a < 3; ++a) {
        if (c.bc_type[a][0] == MRCM_BC_DIRICHLET) geo.dir_lo |= 1 << a;
        if (c.bc_type[a][1] == MRCM_BC_DIRICHLET) geo.dir_hi |= 1 << a;
        geo.glo[a] = c.bc_value[a][0];
        geo.ghi[a] = c.bc_value[a][1];
    }
    double* psum = (double*)(ws + L.psum);
    unsigned long long* mbits = (unsigned long long*)(psum + nsub + 1);
    MRCM_LAUNCH(P, "k_zero_u64", st, k_zero_u64<<<1, 1, 0, st>>>(mbits));
    size_t sm = sizeof(double) * ((size_t)kMaxCells + t.max_m);
    MRCM_LAUNCH(P, "k_reconstruct", st, k_reconstruct<<<nsub, kThreads, sm, st>>>(d.subs, d.faces, d.Ilist, t.NV, (const double*)(ws + L.X), X,
                                             (const double*)(ws + L.coef), (const double*)(ws + L.face_tr),
                                             (const double*)(ws + L.face_beta), K, f, geo, t.n_cells, p, u,
                                             psum, mbits));
    if (!t.has_dirichlet) {
        MRCM_LAUNCH(P, "k_mean", st, k_mean<<<1, kThreads, 0, st>>>(psum, nsub, t.n_cells, psum + nsub));
        MRCM_LAUNCH(P, "k_shift", st, k_shift<<<152 * 4, 256, 0, st>>>(p, t.n_cells, psum + nsub));
    }
    if (mres) cudaMemcpyAsync(mres, mbits, sizeof(double), cudaMemcpyDeviceToDevice, st);
    return (int)cudaGetLastError();
}

}  // namespace mrcm
