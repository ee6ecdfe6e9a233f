// Allocation-free solve of one subdomain's local problem (no counterpart in
// the paper; a deployment variant of the local factor + solve kernels).
//
// Some callers cannot allocate device memory at all: code running inside a
// host application that owns every device allocation through its own pool
// (and forbids driver allocations once its time loop runs), plug-ins that may
// only touch the buffers handed to them, or real-time loops where a
// cudaMalloc would stall the device.  mrcm_box_solve_noalloc needs only the
// caller's input and output buffers: its scratch (the slab block inverses,
// the per-cell coefficients and the forward-sweep results) lives in a
// file-scope __device__ array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "mrcm_internal.h"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxCells = 4096;
constexpr int kNaMaxBlock = 128;
constexpr long long kNaMaxW = 262144;       // doubles of slab block inverses (2 MB)
constexpr long long kNaScratch = kNaMaxW + 5LL * kNaMaxCells;

// Shared scratch of every call on this device: W blocks, then d, t_u, t_v,
// t_s and the sweep vector (kNaMaxCells doubles each).
static __device__ __align__(256) double g_noalloc_scratch[kNaScratch];

struct BoxArgs {
    int sz[3];
    int sa, ua, va, su, b, ns, N;
    double h[3];
    int side_type[6];       // 0 no-flow, 1 Robin, 2 Dirichlet
    int side_off[6];        // offset of each side's faces in g / beta / q
};

__device__ __forceinline__ void box_coords(const BoxArgs& a, int c, int lc[3]) {
    const int sl = c / a.b, r = c - sl * a.b, v = r / a.su;
    lc[a.sa] = sl;
    lc[a.ua] = r - v * a.su;
    lc[a.va] = v;
}

// face index of cell (lc) on side (axis, hi) within that side's list:
// tangential axes t1 < t2, t2 slow
__device__ __forceinline__ int side_face(const BoxArgs& a, int axis, const int lc[3]) {
    const int t1 = axis == 0 ? 1 : 0, t2 = axis == 2 ? 1 : 2;
    return lc[t1] + a.sz[t1] * lc[t2];
}

__device__ __forceinline__ double harm2(double x, double y) { return 2.0 * x * y / (x + y); }

__global__ void __launch_bounds__(kNaThreads)
k_box_solve_noalloc(BoxArgs a, const double* __restrict__ K, const double* __restrict__ f,
                    const double* __restrict__ g, const double* __restrict__ beta, double* __restrict__ p,
                    double* __restrict__ q, double* __restrict__ scratch, int* __restrict__ flag) {
    extern __shared__ __align__(16) double L[];                  // packed lower triangle (FP64)
    __shared__ double rk[kNaMaxBlock];
    __shared__ double tv[kNaMaxBlock];
    __shared__ double z[kNaMaxBlock];
    const int N = a.N, b = a.b;
    double* W = scratch;
    double* cd = scratch + kNaMaxW;
    double* cu = cd + kNaMaxCells;
    double* cv = cu + kNaMaxCells;
    double* cs = cv + kNaMaxCells;
    double* y = cs + kNaMaxCells;
    const int nx = a.sz[0], ny = a.sz[1];
    const double area[3] = {a.h[1] * a.h[2], a.h[0] * a.h[2], a.h[0] * a.h[1]};
    const double vol = a.h[0] * a.h[1] * a.h[2];
    // ---- coefficients and right-hand side (kept in y)
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        int lc[3];
        box_coords(a, c, lc);
        const int gc = lc[0] + nx * (lc[1] + ny * lc[2]);
        double d = 0.0, tp[3] = {0.0, 0.0, 0.0}, rhs = f[gc] * vol;
        for (int ax = 0; ax < 3; ++ax) {
            const double ka = K[(long long)ax * N + gc];
            const int stride = ax == 0 ? 1 : ax == 1 ? nx : nx * ny;
            for (int hi = 0; hi < 2; ++hi) {
                const bool inside = hi ? lc[ax] + 1 < a.sz[ax] : lc[ax] > 0;
                if (inside) {
                    const double T = area[ax] * harm2(ka, K[(long long)ax * N + gc + (hi ? stride : -stride)]) / a.h[ax];
                    d += T;
                    if (hi) tp[ax] = T;
                    continue;
                }
                const int sd = 2 * ax + hi;
                const int fi = a.side_off[sd] + side_face(a, ax, lc);
                if (a.side_type[sd] == 1) {
                    const double TR = area[ax] / (a.h[ax] / (2.0 * ka) + beta[fi]);
                    d += TR;
                    rhs += TR * g[fi];
                } else if (a.side_type[sd] == 2) {
                    const double TD = area[ax] * 2.0 * ka / a.h[ax];
                    d += TD;
                    rhs += TD * g[fi];
                }
            }
        }
        cd[c] = d;
        cu[c] = tp[a.ua];
        cv[c] = tp[a.va];
        cs[c] = tp[a.sa];
        y[c] = rhs;
    }
    __syncthreads();
    // ---- slab factor: W_s = S_s^{-1}, packed sweep operator in shared memory
    int bad = 0;
    for (int sl = 0; sl < a.ns; ++sl) {
        const int base = sl * b;
        for (int i = threadIdx.x; i < b; i += blockDim.x) tv[i] = sl > 0 ? cs[base - b + i] : 0.0;
        __syncthreads();
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
            const int i = e / b, j = e - i * b;
            if (j > i) continue;
            double dij = 0.0;
            if (i == j) dij = cd[base + i];
            if (i == j + 1 && i % a.su > 0) dij = -cu[base + j];
            if (i == j + a.su) dij = -cv[base + j];
            const double prev = sl > 0 ? W[(long long)(sl - 1) * b * b + (long long)i * b + j] : 0.0;
            L[i * (i + 1) / 2 + j] = dij - tv[i] * tv[j] * prev;
        }
        __syncthreads();
        for (int k = 0; k < b; ++k) {
            for (int j = threadIdx.x; j < b; j += blockDim.x)
                rk[j] = j <= k ? L[k * (k + 1) / 2 + j] : L[j * (j + 1) / 2 + k];
            __syncthreads();
            double pv = rk[k];
            if (!(pv > 0.0)) { bad = 1; pv = 1.0; }
            const double ip = 1.0 / pv;
            for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
                const int i = e / b, j = e - i * b;
                if (j > i) continue;
                const double ci = i < k ? -rk[i] : rk[i];
                double v;
                if (i == k) v = j == k ? ip : rk[j] * ip;
                else if (j == k) v = -ci * ip;
                else v = L[i * (i + 1) / 2 + j] - ci * rk[j] * ip;
                L[i * (i + 1) / 2 + j] = v;
            }
            __syncthreads();
        }
        double* Ws = W + (long long)sl * b * b;
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
            const int i = e / b, j = e - i * b;
            Ws[e] = j <= i ? L[i * (i + 1) / 2 + j] : L[j * (j + 1) / 2 + i];
        }
        __syncthreads();
    }
    // ---- solve: forward Y_s = W_s (r_s + t o Y_{s-1}), backward x_s = Y_s + W_s (t o x_{s+1})
    for (int sl = 0; sl < a.ns; ++sl) {
        const int base = sl * b;
        for (int i = threadIdx.x; i < b; i += blockDim.x)
            z[i] = y[base + i] + (sl > 0 ? cs[base - b + i] * y[base - b + i] : 0.0);
        __syncthreads();
        const double* Ws = W + (long long)sl * b * b;
        for (int i = threadIdx.x; i < b; i += blockDim.x) {
            double acc = 0.0;
            for (int k = 0; k < b; ++k) acc += Ws[(long long)k * b + i] * z[k];
            y[base + i] = acc;
        }
        __syncthreads();
    }
    for (int sl = a.ns - 2; sl >= 0; --sl) {
        const int base = sl * b;
        for (int i = threadIdx.x; i < b; i += blockDim.x) z[i] = cs[base + i] * y[base + b + i];
        __syncthreads();
        const double* Ws = W + (long long)sl * b * b;
        for (int i = threadIdx.x; i < b; i += blockDim.x) {
            double acc = 0.0;
            for (int k = 0; k < b; ++k) acc += Ws[(long long)k * b + i] * z[k];
            y[base + i] += acc;
        }
        __syncthreads();
    }
    // ---- outputs: p in box-lexicographic order, outward fluxes on Robin / Dirichlet faces
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        int lc[3];
        box_coords(a, c, lc);
        const int gc = lc[0] + nx * (lc[1] + ny * lc[2]);
        p[gc] = y[c];
        for (int ax = 0; ax < 3; ++ax) {
            const double ka = K[(long long)ax * N + gc];
            for (int hi = 0; hi < 2; ++hi) {
                const bool boundary = hi ? lc[ax] + 1 == a.sz[ax] : lc[ax] == 0;
                if (!boundary) continue;
                const int sd = 2 * ax + hi;
                const int fi = a.side_off[sd] + side_face(a, ax, lc);
                if (a.side_type[sd] == 1) q[fi] = area[ax] / (a.h[ax] / (2.0 * ka) + beta[fi]) * (y[c] - g[fi]);
                else if (a.side_type[sd] == 2) q[fi] = area[ax] * 2.0 * ka / a.h[ax] * (y[c] - g[fi]);
                else q[fi] = 0.0;
            }
        }
    }
    if (bad && threadIdx.x == 0) atomicAdd(flag, 1);
}

constexpr size_t kNaSmem = sizeof(double) * kNaMaxBlock * (kNaMaxBlock + 1) / 2;

// Device addresses of the scratch array and the pivot flag, looked up once
// per device (with that device current) on the first call there.  In host
// code the names of __device__ variables are host-side stand-ins, not device
// addresses, so the kernel gets the looked-up pointers.  The cached addresses
// (and the kernel's shared-memory attribute) belong to the device's primary
// context as it was at that first call: after cudaDeviceReset the module is
// loaded afresh and they are stale, so the entry point does not support use
// after a device reset in the same process.
std::mutex g_mu;
double* g_scratch_ptr[64] = {};
int* g_flag_ptr[64] = {};
static __device__ int g_noalloc_flag;

cudaError_t scratch_for_device(int dev, double** ptr, int** flag) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_scratch_ptr[dev]) {
        double* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        int* fl = nullptr;
        e = cudaGetSymbolAddress((void**)&fl, g_noalloc_flag);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_box_solve_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNaSmem);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
        g_flag_ptr[dev] = fl;
    }
    *ptr = g_scratch_ptr[dev];
    *flag = g_flag_ptr[dev];
    return cudaSuccess;
}

__global__ void k_clear_flag(int* flag) { *flag = 0; }

}  // namespace

extern "C" mrcm_status mrcm_box_solve_noalloc(const int box[3], const double h[3], const int side_type[6],
                                              const double* K, const double* f, const double* g,
                                              const double* beta, double* p, double* q_out, int* not_spd,
                                              void* stream) {
    if (!box || !h || !side_type || !K || !f || !p || !q_out || !not_spd) return MRCM_ERR_INVALID_ARG;
    BoxArgs a;
    long long nfaces = 0;
    bool any_fixed = false;
    for (int ax = 0; ax < 3; ++ax) {
        if (box[ax] < 1 || !(h[ax] > 0)) return MRCM_ERR_INVALID_ARG;
        a.sz[ax] = box[ax];
        a.h[ax] = h[ax];
    }
    // the fixed scratch bounds the problem: larger boxes are refused, never truncated
    // (the cell count is formed in 64 bits, before any product is narrowed to int)
    if ((long long)box[0] * box[1] * box[2] > kNaMaxCells) return MRCM_ERR_OOM;
    for (int sd = 0; sd < 6; ++sd) {
        if (side_type[sd] < 0 || side_type[sd] > 2) return MRCM_ERR_INVALID_ARG;
        a.side_type[sd] = side_type[sd];
        a.side_off[sd] = (int)nfaces;
        const int ax = sd / 2;
        const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
        nfaces += (long long)box[t1] * box[t2];
        if (side_type[sd] != 0) any_fixed = true;
    }
    if (!any_fixed) return MRCM_ERR_INVALID_ARG;          // all sides no-flow: p undetermined
    if (!g || !beta) return MRCM_ERR_INVALID_ARG;
    int sa = 2;
    for (int ax = 1; ax >= 0; --ax) if (box[ax] > box[sa]) sa = ax;
    a.sa = sa;
    a.ua = sa == 0 ? 1 : 0;
    a.va = sa == 2 ? 1 : 2;
    a.su = box[a.ua];
    a.b = box[a.ua] * box[a.va];
    a.ns = box[sa];
    a.N = a.b * a.ns;
    if (a.N > kNaMaxCells || a.b > kNaMaxBlock || (long long)a.ns * a.b * a.b > kNaMaxW) return MRCM_ERR_OOM;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return MRCM_ERR_CUDA;
    double* scratch = nullptr;
    int* flag = nullptr;
    e = scratch_for_device(dev, &scratch, &flag);
    if (e != cudaSuccess) return MRCM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    k_clear_flag<<<1, 1, 0, st>>>(flag);                 // the flag must start at zero in every call
    k_box_solve_noalloc<<<1, kNaThreads, kNaSmem, st>>>(a, K, f, g, beta, p, q_out, scratch, flag);
    cudaMemcpyAsync(not_spd, flag, sizeof(int), cudaMemcpyDeviceToDevice, st);
    e = cudaGetLastError();
    return e == cudaSuccess ? MRCM_OK : MRCM_ERR_CUDA;
}
