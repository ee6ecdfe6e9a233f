// Two-phase IMPES transport with a skipping constant (Sec. "The fine grid
// transport solver", Eq. transporte_discreto, Eq. flux_disc_up, Eq. CFL,
// Alg. overview-code).
//
// Water saturation S (time rescaled by the porosity), total mobility
// lambda(S) = S^2/mu_w + (1-S)^2/mu_o, fractional flow
// phi(S) = M S^2 / (M S^2 + (1-S)^2), M = mu_o/mu_w.  Every C transport steps
// the Darcy problem is solved again with K_eff = lambda(S) K (the MRCM solve
// and its mean velocity post-processing, which makes the velocity
// conservative on the fine grid); in between, the velocity and the step stay
// frozen.  Transport step, the conservative upwind finite-volume update in the
// paper's compensated form (the frozen velocity's divergence is removed with
// the cell's own phi, which keeps the scheme monotone):
//   S_c <- S_c - (dt/V) sum_faces (phi_f - phi_c) q_f + dt max(f_c, 0) (1 - phi_c),
// q_f the outward integrated flux, phi_f of the upwind cell, no flux through
// the (no-flow) walls.  dt = cfl min(h) / (phi'_max max|u|) (Eq. CFL, with
// phi'_max the maximum of phi' over S = k/1000, a bound over [0, 1]).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "mrcm_internal.h"

namespace mrcm {
namespace {

constexpr int kTThreads = 256;

struct TGeo {
    int n[3];
    double area[3];
    double inv_vol;
};

__device__ __forceinline__ double frac_flow(double S, double M) {
    const double w = M * S * S;
    return w / (w + (1.0 - S) * (1.0 - S));
}

// K_eff[a][c] = lambda(S_c) K[a][c]
__global__ void __launch_bounds__(kTThreads)
k_mobility(const double* __restrict__ K, const double* __restrict__ S, double mu_w, double mu_o,
           double* __restrict__ Ke, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double s = S[c];
        const double lam = s * s / mu_w + (1.0 - s) * (1.0 - s) / mu_o;
        Ke[c] = lam * K[c];
        Ke[n + c] = lam * K[n + c];
        Ke[2 * n + c] = lam * K[2 * n + c];
    }
}

// max |u| over all face entries (atomicMax on the bits of a non-negative double)
__global__ void __launch_bounds__(kTThreads)
k_umax(const double* __restrict__ u, long long n, unsigned long long* __restrict__ bits) {
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(u[i]));
    __shared__ double red[kTThreads];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(bits, (unsigned long long)__double_as_longlong(red[0]));
}

// sc[0] = max|u| bits, sc[1] = dt, sc[2] = t
__global__ void k_dt(double* sc, double num) {
    const double umax = sc[0];
    sc[1] = umax > 0.0 ? num / umax : 0.0;
}

__global__ void k_tadd(double* sc) { sc[2] += sc[1]; }

__global__ void k_zero_doubles(double* p, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0.0;
}

// phi(S) of every cell (one FP64 division each), read by the step for the
// upwind faces
__global__ void __launch_bounds__(kTThreads)
k_frac_flow(const double* __restrict__ S, double* __restrict__ phi, double M, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        phi[c] = frac_flow(S[c], M);
}

// One upwind step S_in -> S_out with the frozen, single-valued velocity u and
// the cells' phi (and phi of S_out for the next step); cell coordinates in
// 32-bit arithmetic (n < 2^31 cells).
__global__ void __launch_bounds__(kTThreads)
k_transport_step(const double* __restrict__ S, double* __restrict__ Sn, const double* __restrict__ phi,
                 double* __restrict__ phin, const double* __restrict__ u, const double* __restrict__ f,
                 const double* __restrict__ sc, TGeo g, double M) {
    const int n = g.n[0] * g.n[1] * g.n[2];
    const int nxy = g.n[0] * g.n[1];
    const int stride[3] = {1, g.n[0], nxy};
    const double dt = sc[1];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int k = c / nxy, r = c - k * nxy, j = r / g.n[0];
        const int co[3] = {r - j * g.n[0], j, k};
        const double phic = phi[c];
        double acc = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (co[a] + 1 < g.n[a]) {                          // face on the +a side
                const double q = u[(long long)(2 * a + 1) * n + c] * g.area[a];
                const double phf = q >= 0.0 ? phic : phi[c + stride[a]];
                acc -= (phf - phic) * q;
            }
            if (co[a] > 0) {                                   // face on the -a side
                const double q = -(u[(long long)(2 * a) * n + c] * g.area[a]);
                const double phf = q >= 0.0 ? phic : phi[c - stride[a]];
                acc -= (phf - phic) * q;
            }
        }
        const double sn = S[c] + dt * g.inv_vol * acc + dt * fmax(f[c], 0.0) * (1.0 - phic);
        Sn[c] = sn;
        phin[c] = frac_flow(sn, M);                            // phi of the next step
    }
}

double frac_flow_slope_max(double M) {
    double mx = 0.0;
    for (int k = 0; k <= 1000; ++k) {
        const double S = k / 1000.0;
        const double d = M * S * S + (1.0 - S) * (1.0 - S);
        mx = std::max(mx, 2.0 * M * S * (1.0 - S) / (d * d));
    }
    return mx;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct TLayout {
    size_t ke, u, upp, p, X, S2, phi, phi2, sc, total;
};

TLayout transport_layout(const Tables& t) {
    TLayout L;
    const size_t n = (size_t)t.n_cells;
    size_t o = 0;
    L.ke = o; o = al256(o + 3 * n * sizeof(double));
    L.u = o; o = al256(o + 6 * n * sizeof(double));
    L.upp = o; o = al256(o + 6 * n * sizeof(double));
    L.p = o; o = al256(o + n * sizeof(double));
    L.X = o; o = al256(o + std::max<size_t>(2 * (size_t)t.NV, 1) * sizeof(double));
    L.S2 = o; o = al256(o + n * sizeof(double));
    L.phi = o; o = al256(o + n * sizeof(double));
    L.phi2 = o; o = al256(o + n * sizeof(double));
    L.sc = o; o = al256(o + 8 * sizeof(double));
    L.total = o;
    return L;
}

}  // namespace
}  // namespace mrcm

extern "C" {

mrcm_status mrcm_transport_query(const mrcm_handle* h, size_t* bytes) {
    if (!h || !bytes) return MRCM_ERR_INVALID_ARG;
    *bytes = mrcm::transport_layout(h->t).total;
    return MRCM_OK;
}

mrcm_status mrcm_impes(mrcm_handle* h, const double* K, const double* f, double* S, double mu_w, double mu_o,
                       double cfl, int C, int n_steps, double* t_out, void* tws, size_t tws_bytes, void* ws,
                       size_t ws_bytes, void* stream) {
    if (!h) return MRCM_ERR_INVALID_ARG;
    const mrcm::Tables& t = h->t;
    if (!K || !f || !S || !tws || !ws || !(mu_w > 0) || !(mu_o > 0) || !(cfl > 0) || C < 1 || n_steps < 0) {
        h->err = "mrcm_impes: bad argument";
        return MRCM_ERR_INVALID_ARG;
    }
    if (t.has_dirichlet) { h->err = "mrcm_impes: the transport step takes no-flow walls only"; return MRCM_ERR_NOT_IMPLEMENTED; }
    if (t.n_cells >= (1LL << 31) / 6) { h->err = "mrcm_impes: grid too large for 32-bit face indexing"; return MRCM_ERR_NOT_IMPLEMENTED; }
    const mrcm::TLayout L = mrcm::transport_layout(t);
    if (tws_bytes < L.total) { h->err = "transport workspace smaller than mrcm_transport_query"; return MRCM_ERR_OOM; }
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)tws;
    double* Ke = (double*)(w + L.ke);
    double* u = (double*)(w + L.u);
    double* upp = (double*)(w + L.upp);
    double* p = (double*)(w + L.p);
    double* X = (double*)(w + L.X);
    double* S2 = (double*)(w + L.S2);
    double* phi = (double*)(w + L.phi);
    double* phi2 = (double*)(w + L.phi2);
    double* sc = (double*)(w + L.sc);         // [0] max|u| bits, [1] dt, [2] t, [3] mass residual
    const long long n = t.n_cells;
    const double M = mu_o / mu_w;
    const double hmin = std::min(t.cfg.hx, std::min(t.cfg.hy, t.cfg.hz));
    const double num = cfl * hmin / mrcm::frac_flow_slope_max(M);
    mrcm::TGeo g;
    g.n[0] = t.cfg.nx; g.n[1] = t.cfg.ny; g.n[2] = t.cfg.nz;
    g.area[0] = t.cfg.hy * t.cfg.hz; g.area[1] = t.cfg.hx * t.cfg.hz; g.area[2] = t.cfg.hx * t.cfg.hy;
    g.inv_vol = 1.0 / (t.cfg.hx * t.cfg.hy * t.cfg.hz);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = sms * 8;
    MRCM_LAUNCH(h->prof, "k_zero_int", st, mrcm::k_zero_doubles<<<1, 32, 0, st>>>(sc, 8));
    double* cur = S;
    double* nxt = S2;
    for (int step = 0; step < n_steps; ++step) {
        if (step % C == 0) {
            MRCM_LAUNCH(h->prof, "k_mobility", st, mrcm::k_mobility<<<grid, mrcm::kTThreads, 0, st>>>(K, cur, mu_w, mu_o, Ke, n));
            mrcm_status rs = mrcm_solve(h, Ke, f, X, p, u, sc + 3, ws, ws_bytes, stream, 0);
            if (rs != MRCM_OK) return rs;
            rs = mrcm_postprocess_velocity(h, u, upp, sc + 3, ws, stream);
            if (rs != MRCM_OK) return rs;
            MRCM_LAUNCH(h->prof, "k_zero_int", st, mrcm::k_zero_doubles<<<1, 32, 0, st>>>(sc, 1));
            MRCM_LAUNCH(h->prof, "k_cfl", st, mrcm::k_umax<<<grid, mrcm::kTThreads, 0, st>>>(upp, 6 * n, (unsigned long long*)sc));
            MRCM_LAUNCH(h->prof, "k_cfl", st, mrcm::k_dt<<<1, 1, 0, st>>>(sc, num));
        }
        if (step == 0)
            MRCM_LAUNCH(h->prof, "k_frac_flow", st, mrcm::k_frac_flow<<<grid, mrcm::kTThreads, 0, st>>>(cur, phi, M, n));
        MRCM_LAUNCH(h->prof, "k_transport_step", st, mrcm::k_transport_step<<<grid, mrcm::kTThreads, 0, st>>>(cur, nxt, phi, phi2, upp, f, sc, g, M));
        std::swap(phi, phi2);
        MRCM_LAUNCH(h->prof, "k_tadd", st, mrcm::k_tadd<<<1, 1, 0, st>>>(sc));
        std::swap(cur, nxt);
    }
    if (cur != S) cudaMemcpyAsync(S, cur, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    if (t_out) cudaMemcpyAsync(t_out, sc + 2, sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (cudaGetLastError() != cudaSuccess) { h->err = "mrcm_impes: launch failed"; return MRCM_ERR_CUDA; }
    return MRCM_OK;
}

}  // extern "C"
