// Learned warm start for the local solves (no counterpart in the paper):
// a small 3-D convolutional network maps a subdomain's log-permeability and
// the Robin data of one basis function to a guess of that P-MBF's pressure,
// which seeds an FP32 conjugate-gradient solve of the local system.
//
// Network: L layers of 3x3x3 'same' convolutions (zero padding), leaky ReLU
// (slope 1/100) after every layer but the last, a logistic output (P-MBFs lie in [0, 1] by the
// maximum principle).  Weights are held in FP32 (master, Adam moments) and
// used in BF16 by the forward and backward-data convolutions; all
// accumulation is FP32.  Activations are [batch][channel][z][y][x] FP32.
//
// Training data come from the method itself: after mrcm_solve_mbf, every
// P-MBF column of every subdomain with the network's box shape becomes one
// sample (inputs: log Kx / 4, log Kz / 4, the Robin data of the basis on the cells
// next to its faces, a mask of all Robin faces; target: the column).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mrcm_internal.h"

struct mrcm_net {
    int in_ch, hidden, layers, D, H, W, S;
    std::vector<int> cin, cout;          // per layer
    std::vector<long long> w_off, b_off; // offsets (floats) into the parameter vector
    long long P = 0;                     // parameter count
    std::vector<long long> act_off;      // offsets (floats per sample) of stored activations
    long long act_per_sample = 0;
    int max_ch = 0;
    bool mma_ok = false;                 // 32 -> 32 layers take the tensor-core forward (its shared memory fits)
};

namespace mrcm {
namespace {

constexpr int kNetThreads = 256;
constexpr int kMaxCh = 32;
constexpr float kLeak = 0.01f;       // leaky-ReLU slope
constexpr float kLogKScale = 0.25f;  // log K channels are scaled by 1/4

struct ConvShape { int D, H, W, S; };

__device__ __forceinline__ int tap_offset_ok(const ConvShape& sh, int p, int tap, int* q) {
    const int z = p / (sh.H * sh.W), r = p - z * sh.H * sh.W, y = r / sh.W, x = r - y * sh.W;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int zz = z + dz, yy = y + dy, xx = x + dx;
    if (zz < 0 || zz >= sh.D || yy < 0 || yy >= sh.H || xx < 0 || xx >= sh.W) return 0;
    *q = (zz * sh.H + yy) * sh.W + xx;
    return 1;
}

// out[b][co][p] = act( bias[co] + sum_ci sum_tap w[co][ci][tap] in[b][ci][p + tap] )
// Weights come from the BF16 copy; the CTA stages them as FP32 [ci][tap][co].
// mode 0: leaky ReLU, 1: logistic, 2: none.  One CTA per sample.
template <int CO>   // accumulators per thread: kMaxCh, or 1 for the one-channel output layer
__global__ void __launch_bounds__(kNetThreads)
k_conv_forward(ConvShape sh, int Cin, int Cout, const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
               const float* __restrict__ in, float* __restrict__ out, int mode) {
    extern __shared__ __align__(16) float sm[];
    float* xin = sm;                                   // Cin x S
    float* ws = xin + Cin * sh.S;                      // Cin x 27 x Cout
    const int b = blockIdx.x;
    const float* ib = in + (long long)b * Cin * sh.S;
    for (int e = threadIdx.x; e < Cin * sh.S; e += blockDim.x) xin[e] = ib[e];
    for (int e = threadIdx.x; e < Cout * Cin * 27; e += blockDim.x) {
        const int co = e / (Cin * 27), r = e - co * Cin * 27, ci = r / 27, tap = r - ci * 27;
        ws[(ci * 27 + tap) * Cout + co] = __bfloat162float(w[e]);
    }
    __syncthreads();
    float* ob = out + (long long)b * Cout * sh.S;
    for (int p = threadIdx.x; p < sh.S; p += blockDim.x) {
        float acc[CO];
#pragma unroll
        for (int co = 0; co < CO; ++co) acc[co] = 0.0f;
        for (int tap = 0; tap < 27; ++tap) {
            int q;
            if (!tap_offset_ok(sh, p, tap, &q)) continue;
            for (int ci = 0; ci < Cin; ++ci) {
                const float x = xin[ci * sh.S + q];
                const float* wr = ws + (ci * 27 + tap) * Cout;
#pragma unroll
                for (int co = 0; co < CO; ++co)
                    if (co < Cout) acc[co] = fmaf(wr[co], x, acc[co]);
            }
        }
#pragma unroll
        for (int co = 0; co < CO; ++co) {
            if (co >= Cout) break;
            float v = acc[co] + bias[co];
            if (mode == 0) v = v > 0.0f ? v : kLeak * v;
            else if (mode == 1) v = 1.0f / (1.0f + __expf(-v));
            ob[(long long)co * sh.S + p] = v;
        }
    }
}

// The same forward for a 32 -> 32 channel layer as an implicit GEMM on the BF16
// tensor cores: out[co][p] = bias[co] + sum_k A[co][k] B[k][p] with k = tap 32 + ci,
// A = the BF16 weights (exact in BF16), B[k][p] = in[ci][p + tap] cut into three BF16
// pieces x = x1 + x2 + x3 (x1 the rounded value, x2 and x3 the rounded remainders, which
// carry x to FP32 accuracy); mma.sync m16n8k16 with FP32 accumulation (a BF16 x BF16
// product is exact in FP32), so the result matches the FP32 direct convolution to FP32
// rounding.  The sample sits in shared memory with a zero halo, channels innermost
// ([padded voxel][32] FP32), the weights as [co][k] BF16 pairs; one CTA per SM walks the
// samples, staging the weights once.  Each of 16 warps takes up to 4 tiles of 8 voxels at a time.
constexpr int kMmaCh = 32;
constexpr int kMmaTiles = 4;
constexpr int kMmaThreads = 512;
size_t conv_mma_smem(const ConvShape& sh) {
    return sizeof(float) * (size_t)(sh.D + 2) * (sh.H + 2) * (sh.W + 2) * kMmaCh + sizeof(uint32_t) * kMmaCh * 27 * kMmaCh / 2;
}
__device__ __forceinline__ void mma_bf16_16816(float d[4], const uint32_t a[4], const uint32_t b[2]) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t*>(&h); }
// v = v1 + v2 + v3, each a BF16 pair (low half = v.x)
__device__ __forceinline__ void split3_bf16(float2 v, uint32_t& p1, uint32_t& p2, uint32_t& p3) {
    const __nv_bfloat162 h1 = __float22bfloat162_rn(v);
    const float2 f1 = __bfloat1622float2(h1);
    const float2 r1 = make_float2(v.x - f1.x, v.y - f1.y);
    const __nv_bfloat162 h2 = __float22bfloat162_rn(r1);
    const float2 f2 = __bfloat1622float2(h2);
    const float2 r2 = make_float2(r1.x - f2.x, r1.y - f2.y);
    p1 = bf2_bits(h1);
    p2 = bf2_bits(h2);
    p3 = bf2_bits(__float22bfloat162_rn(r2));
}
__global__ void __launch_bounds__(kMmaThreads, 1)
k_conv_forward_mma(ConvShape sh, int batch, const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
                   const float* __restrict__ in, float* __restrict__ out, int mode) {
    extern __shared__ __align__(16) unsigned char smc[];
    const int Hp = sh.H + 2, Wp = sh.W + 2, Sp = (sh.D + 2) * Hp * Wp;
    constexpr int KW = 27 * kMmaCh / 2;                                 // BF16 pairs per weight row
    float* xs = reinterpret_cast<float*>(smc);                          // [Sp][32]
    uint32_t* wsm = reinterpret_cast<uint32_t*>(xs + (size_t)Sp * kMmaCh);   // [co][KW]
    for (int e = threadIdx.x; e < kMmaCh * KW; e += blockDim.x) {
        const int co = e / KW, r = e - co * KW, tap = r / (kMmaCh / 2), cp = r - tap * (kMmaCh / 2);
        const __nv_bfloat16 lo = w[(co * kMmaCh + 2 * cp) * 27 + tap], hi = w[(co * kMmaCh + 2 * cp + 1) * 27 + tap];
        wsm[e] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
    }
    for (int e = threadIdx.x; e < Sp * kMmaCh; e += blockDim.x) xs[e] = 0.0f;   // the halo stays zero
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int nwarps = blockDim.x >> 5;
    const int ntiles = (sh.S + 7) / 8;
    for (int b = blockIdx.x; b < batch; b += gridDim.x) {
        __syncthreads();                                                // previous sample done with xs
        const float* ib = in + (long long)b * kMmaCh * sh.S;
        for (int e = threadIdx.x; e < kMmaCh * sh.S; e += blockDim.x) {
            const int ci = e / sh.S, p = e - ci * sh.S;
            const int z = p / (sh.H * sh.W), r = p - z * sh.H * sh.W, y = r / sh.W, x = r - y * sh.W;
            xs[(((z + 1) * Hp + y + 1) * Wp + x + 1) * kMmaCh + ci] = ib[e];
        }
        __syncthreads();
        for (int nt0 = warp; nt0 < ntiles; nt0 += nwarps * kMmaTiles) {
            float acc[kMmaTiles][2][4];
            int pvb[kMmaTiles];
#pragma unroll
            for (int j = 0; j < kMmaTiles; ++j) {
                const int p = (nt0 + nwarps * j) * 8 + g;
                int pv = (Hp + 1) * Wp + 1;                             // padding columns: voxel 0 (all 27
                                                                        // neighbours in range), discarded
                if (nt0 + nwarps * j < ntiles && p < sh.S) {
                    const int z = p / (sh.H * sh.W), r = p - z * sh.H * sh.W, y = r / sh.W, x = r - y * sh.W;
                    pv = ((z + 1) * Hp + y + 1) * Wp + x + 1;
                }
                pvb[j] = pv;
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[j][mt][q] = 0.0f;
            }
#pragma unroll 1
            for (int tap = 0; tap < 27; ++tap) {
                const int toff = ((tap / 9 - 1) * Hp + (tap / 3) % 3 - 1) * Wp + tap % 3 - 1;
#pragma unroll
                for (int kc = 0; kc < 2; ++kc) {
                    const int kw = tap * (kMmaCh / 2) + kc * 8 + t;
                    uint32_t a[2][4];
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        const int r0 = mt * 16 + g;
                        a[mt][0] = wsm[r0 * KW + kw];
                        a[mt][1] = wsm[(r0 + 8) * KW + kw];
                        a[mt][2] = wsm[r0 * KW + kw + 4];
                        a[mt][3] = wsm[(r0 + 8) * KW + kw + 4];
                    }
#pragma unroll
                    for (int j = 0; j < kMmaTiles; ++j) {
                        if (nt0 + nwarps * j >= ntiles) break;          // warp-uniform
                        const float* xp = xs + (pvb[j] + toff) * kMmaCh + kc * 16 + 2 * t;
                        uint32_t b1[2], b2[2], b3[2];
                        split3_bf16(*reinterpret_cast<const float2*>(xp), b1[0], b2[0], b3[0]);
                        split3_bf16(*reinterpret_cast<const float2*>(xp + 8), b1[1], b2[1], b3[1]);
#pragma unroll
                        for (int mt = 0; mt < 2; ++mt) {
                            mma_bf16_16816(acc[j][mt], a[mt], b3);      // smallest pieces first
                            mma_bf16_16816(acc[j][mt], a[mt], b2);
                            mma_bf16_16816(acc[j][mt], a[mt], b1);
                        }
                    }
                }
            }
            float* ob = out + (long long)b * kMmaCh * sh.S;
#pragma unroll
            for (int j = 0; j < kMmaTiles; ++j) {
                const int nt = nt0 + nwarps * j;
                if (nt >= ntiles) break;
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int co = mt * 16 + g + (q >> 1) * 8, p = nt * 8 + 2 * t + (q & 1);
                        if (p >= sh.S) continue;
                        float v = acc[j][mt][q] + bias[co];
                        if (mode == 0) v = v > 0.0f ? v : kLeak * v;
                        else if (mode == 1) v = 1.0f / (1.0f + __expf(-v));
                        ob[(long long)co * sh.S + p] = v;
                    }
            }
        }
    }
}

// grad_in[b][ci][q] = sum_co sum_tap w[co][ci][tap] g[b][co][q - tap]  (backward data),
// multiplied by the derivative of the producing layer's leaky ReLU when relu_in.
__global__ void __launch_bounds__(kNetThreads)
k_conv_backward_data(ConvShape sh, int Cin, int Cout, const __nv_bfloat16* __restrict__ w,
                     const float* __restrict__ g, const float* __restrict__ act_in, float* __restrict__ gin,
                     int relu_in) {
    extern __shared__ __align__(16) float sm[];
    float* gs = sm;                                    // Cout x S
    float* ws = gs + Cout * sh.S;                      // Cout x 27 x Cin
    const int b = blockIdx.x;
    const float* gb = g + (long long)b * Cout * sh.S;
    for (int e = threadIdx.x; e < Cout * sh.S; e += blockDim.x) gs[e] = gb[e];
    for (int e = threadIdx.x; e < Cout * Cin * 27; e += blockDim.x) {
        const int co = e / (Cin * 27), r = e - co * Cin * 27, ci = r / 27, tap = r - ci * 27;
        ws[(co * 27 + tap) * Cin + ci] = __bfloat162float(w[e]);
    }
    __syncthreads();
    float* ob = gin + (long long)b * Cin * sh.S;
    const float* ab = act_in + (long long)b * Cin * sh.S;
    for (int q = threadIdx.x; q < sh.S; q += blockDim.x) {
        float acc[kMaxCh];
#pragma unroll
        for (int ci = 0; ci < kMaxCh; ++ci) acc[ci] = 0.0f;
        for (int tap = 0; tap < 27; ++tap) {
            int p;
            // output p with p + tap == q: p = q - tap, i.e. the mirrored tap from q
            if (!tap_offset_ok(sh, q, 26 - tap, &p)) continue;
            for (int co = 0; co < Cout; ++co) {
                const float gv = gs[co * sh.S + p];
                const float* wr = ws + (co * 27 + tap) * Cin;
#pragma unroll
                for (int ci = 0; ci < kMaxCh; ++ci)
                    if (ci < Cin) acc[ci] = fmaf(wr[ci], gv, acc[ci]);
            }
        }
#pragma unroll
        for (int ci = 0; ci < kMaxCh; ++ci) {
            if (ci >= Cin) break;
            float v = acc[ci];
            if (relu_in && !(ab[(long long)ci * sh.S + q] > 0.0f)) v *= kLeak;
            ob[(long long)ci * sh.S + q] = v;
        }
    }
}

// grad_w[co][ci][tap] = sum_b sum_p g[b][co][p] in[b][ci][p + tap]; grad_b[co] = sum g.
// One CTA per (co, ci); fixed-order block reductions (deterministic).
__global__ void __launch_bounds__(kNetThreads)
k_conv_backward_weights(ConvShape sh, int Cin, int Cout, int batch, const float* __restrict__ g,
                        const float* __restrict__ in, float* __restrict__ gw, float* __restrict__ gbias) {
    const int co = blockIdx.x / Cin, ci = blockIdx.x - (blockIdx.x / Cin) * Cin;
    float acc[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) acc[t] = 0.0f;
    float accb = 0.0f;
    for (int e = threadIdx.x; e < batch * sh.S; e += blockDim.x) {
        const int b = e / sh.S, p = e - b * sh.S;
        const float gv = g[((long long)b * Cout + co) * sh.S + p];
        accb += gv;
        const float* ib = in + ((long long)b * Cin + ci) * sh.S;
#pragma unroll
        for (int t = 0; t < 27; ++t) {
            int q;
            if (tap_offset_ok(sh, p, t, &q)) acc[t] = fmaf(gv, ib[q], acc[t]);
        }
    }
    __shared__ float red[kNetThreads];
    for (int t = 0; t < 28; ++t) {
        red[threadIdx.x] = t < 27 ? acc[t] : accb;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (t < 27) gw[((long long)co * Cin + ci) * 27 + t] = red[0];
            else if (ci == 0) gbias[co] = red[0];
        }
        __syncthreads();
    }
}

// Loss over the batch and its gradient with respect to the logistic output's
// pre-activation.  Without weights the pressure MSE, mean((y - t)^2); with
// per-cell weights w (the sum of T_R^2 over the cell's Robin faces) the
// squared face-flux errors are added, T_R (y_c - t_c) being the error of the
// outward flux through a face of the cell: mean((1 + w) (y - t)^2), whose
// derivative is 2 (1 + w) (y - t) y (1 - y) / n.
__global__ void __launch_bounds__(kNetThreads)
k_mse_loss(int n, const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ w,
           float* __restrict__ g, float* __restrict__ partial) {
    __shared__ float red[kNetThreads];
    float acc = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        const float wt = w ? 1.0f + w[i] : 1.0f;
        acc += wt * d * d;
        g[i] = 2.0f * wt * d * y[i] * (1.0f - y[i]) / (float)n;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(int n, int count, const float* __restrict__ partial, float* __restrict__ loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.0f;
        for (int i = 0; i < count; ++i) s += partial[i];
        *loss = s / (float)n;
    }
}

// Adam on the FP32 master weights, then the BF16 copy.
__global__ void k_adam(long long P, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, __nv_bfloat16* __restrict__ wb, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wb[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void k_to_bf16(long long P, const float* __restrict__ w, __nv_bfloat16* __restrict__ wb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16_rn(w[i]);
}

// splitmix64 (Steele, Lea and Flood, 2014) as a counter-based generator:
// value i of stream `seed` is the mix of seed + (i + 1) * golden gamma.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// He-normal weights (Box-Muller on two splitmix64 uniforms), zero biases.
__global__ void k_init(long long P, float* __restrict__ w, const unsigned char* __restrict__ is_bias,
                       const float* __restrict__ stddev, unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
        if (is_bias[i]) { w[i] = 0.0f; continue; }
        const unsigned long long a = splitmix64(seed + 0x9e3779b97f4a7c15ULL * (2 * (unsigned long long)i + 1));
        const unsigned long long c = splitmix64(seed + 0x9e3779b97f4a7c15ULL * (2 * (unsigned long long)i + 2));
        const double u1 = ((a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((c >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double nrm = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
        w[i] = (float)(nrm * stddev[i]);
    }
}

__global__ void k_zero_f(long long n, float* __restrict__ x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = 0.0f;
}

size_t conv_smem(int C1, int C2, int S) { return sizeof(float) * ((size_t)C1 * S + (size_t)C1 * C2 * 27); }

}  // namespace
}  // namespace mrcm

using mrcm::ConvShape;

namespace {

// parameter state layout (floats): master P | m P | v P | bf16 copy (P/2 floats, rounded up)
long long state_floats(const mrcm_net* n) { return 3 * n->P + (n->P + 1) / 2 + 1; }

struct NetPtrs {
    float* w; float* m; float* v; __nv_bfloat16* wb;
};

NetPtrs net_ptrs(const mrcm_net* n, const float* state) {
    NetPtrs p;
    p.w = const_cast<float*>(state);
    p.m = p.w + n->P;
    p.v = p.m + n->P;
    p.wb = reinterpret_cast<__nv_bfloat16*>(p.v + n->P);
    return p;
}

// Workspace per sample: stored activations (input copy not needed: given),
// then two gradient buffers of max_ch x S, plus loss partials.
size_t net_ws_bytes(const mrcm_net* n, int batch) {
    const size_t per = (size_t)n->act_per_sample + 2 * (size_t)n->max_ch * n->S;
    return sizeof(float) * (per * (size_t)batch + 1024 + (size_t)n->P) + 256;
}

void forward(const mrcm_net* n, const NetPtrs& p, const float* x, int batch, float* acts, cudaStream_t st) {
    ConvShape sh{n->D, n->H, n->W, n->S};
    const float* in = x;
    for (int l = 0; l < n->layers; ++l) {
        float* out = acts + (long long)batch * n->act_off[l];
        const int mode = l + 1 == n->layers ? 1 : 0;
        if (n->cin[l] == mrcm::kMmaCh && n->cout[l] == mrcm::kMmaCh && n->mma_ok) {
            int dev = 0, sms = 1;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            mrcm::k_conv_forward_mma<<<std::max(1, std::min(batch, sms)), mrcm::kMmaThreads, mrcm::conv_mma_smem(sh), st>>>(
                sh, batch, p.wb + n->w_off[l], p.w + n->b_off[l], in, out, mode);
        } else {
            const size_t sm = mrcm::conv_smem(n->cin[l], n->cout[l], n->S);
            if (n->cout[l] == 1)
                mrcm::k_conv_forward<1><<<batch, mrcm::kNetThreads, sm, st>>>(sh, n->cin[l], n->cout[l], p.wb + n->w_off[l],
                                                                             p.w + n->b_off[l], in, out, mode);
            else
                mrcm::k_conv_forward<mrcm::kMaxCh><<<batch, mrcm::kNetThreads, sm, st>>>(sh, n->cin[l], n->cout[l],
                    p.wb + n->w_off[l], p.w + n->b_off[l], in, out, mode);
        }
        in = out;
    }
}

// loss and gradient of the parameters into `grad` (P floats)
void backward(const mrcm_net* n, const NetPtrs& p, const float* x, const float* target, const float* weight,
              int batch, float* acts, float* gbuf0, float* gbuf1, float* grad, float* partial, float* loss,
              cudaStream_t st) {
    ConvShape sh{n->D, n->H, n->W, n->S};
    const int L = n->layers;
    const float* y = acts + (long long)batch * n->act_off[L - 1];
    const int nout = batch * n->S;
    const int nb = 128;
    mrcm::k_mse_loss<<<nb, mrcm::kNetThreads, 0, st>>>(nout, y, target, weight, gbuf0, partial);
    mrcm::k_sum_partials<<<1, 32, 0, st>>>(nout, nb, partial, loss);
    float* g = gbuf0;
    float* gnext = gbuf1;
    for (int l = L - 1; l >= 0; --l) {
        const float* in = l == 0 ? x : acts + (long long)batch * n->act_off[l - 1];
        mrcm::k_conv_backward_weights<<<n->cout[l] * n->cin[l], mrcm::kNetThreads, 0, st>>>(
            sh, n->cin[l], n->cout[l], batch, g, in, grad + n->w_off[l], grad + n->b_off[l]);
        if (l > 0) {
            const size_t sm = mrcm::conv_smem(n->cout[l], n->cin[l], n->S);
            mrcm::k_conv_backward_data<<<batch, mrcm::kNetThreads, sm, st>>>(sh, n->cin[l], n->cout[l],
                                                                           p.wb + n->w_off[l], g, in, gnext, 1);
            float* t = g; g = gnext; gnext = t;
        }
    }
}

}  // namespace

extern "C" {

mrcm_status mrcm_net_create(int in_channels, int hidden, int layers, int D, int H, int W, mrcm_net** out) {
    if (!out) return MRCM_ERR_INVALID_ARG;
    *out = nullptr;
    if (in_channels < 1 || in_channels > mrcm::kMaxCh || hidden < 1 || hidden > mrcm::kMaxCh || layers < 2 ||
        layers > 16 || D < 1 || H < 1 || W < 1 || (long long)D * H * W > 4096)
        return MRCM_ERR_INVALID_ARG;
    mrcm_net* n = new mrcm_net();
    n->in_ch = in_channels; n->hidden = hidden; n->layers = layers;
    n->D = D; n->H = H; n->W = W; n->S = D * H * W;
    long long off = 0, aoff = 0;
    for (int l = 0; l < layers; ++l) {
        const int ci = l == 0 ? in_channels : hidden;
        const int co = l + 1 == layers ? 1 : hidden;
        n->cin.push_back(ci);
        n->cout.push_back(co);
        n->w_off.push_back(off); off += (long long)co * ci * 27;
        n->b_off.push_back(off); off += co;
        n->act_off.push_back(aoff); aoff += (long long)co * n->S;
        n->max_ch = std::max(n->max_ch, std::max(ci, co));
    }
    n->P = off;
    n->act_per_sample = aoff;
    const size_t sm = std::max(mrcm::conv_smem(hidden, hidden, n->S), mrcm::conv_smem(in_channels, hidden, n->S));
    if (sm > 227 * 1024) { delete n; return MRCM_ERR_NOT_IMPLEMENTED; }
    cudaFuncSetAttribute(mrcm::k_conv_forward<mrcm::kMaxCh>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(mrcm::k_conv_forward<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    {
        const size_t smm = mrcm::conv_mma_smem(mrcm::ConvShape{n->D, n->H, n->W, n->S});
        n->mma_ok = smm <= 227 * 1024 &&
                    cudaFuncSetAttribute(mrcm::k_conv_forward_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smm) == cudaSuccess;
        cudaGetLastError();
    }
    cudaFuncSetAttribute(mrcm::k_conv_backward_data, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    *out = n;
    return MRCM_OK;
}

mrcm_status mrcm_net_query(const mrcm_net* n, int batch, size_t* params, size_t* state_floats_out,
                           size_t* ws_bytes) {
    if (!n || batch < 1) return MRCM_ERR_INVALID_ARG;
    if (params) *params = (size_t)n->P;
    if (state_floats_out) *state_floats_out = (size_t)state_floats(n);
    if (ws_bytes) *ws_bytes = net_ws_bytes(n, batch);
    return MRCM_OK;
}

mrcm_status mrcm_net_init(mrcm_net* n, float* state, unsigned long long seed, void* stream) {
    if (!n || !state) return MRCM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    NetPtrs p = net_ptrs(n, state);
    // He-normal standard deviations per parameter, uploaded once (small)
    std::vector<float> sd(n->P, 0.0f);
    std::vector<unsigned char> isb(n->P, 0);
    for (int l = 0; l < n->layers; ++l) {
        // He-normal; the output layer starts 10x smaller so that the logistic
        // output is not saturated before training
        const float s = std::sqrt(2.0f / (27.0f * n->cin[l])) * (l + 1 == n->layers ? 0.1f : 1.0f);
        for (long long i = n->w_off[l]; i < n->b_off[l]; ++i) sd[i] = s;
        for (long long i = n->b_off[l]; i < n->b_off[l] + n->cout[l]; ++i) isb[i] = 1;
    }
    float* dsd = nullptr;
    unsigned char* disb = nullptr;
    // the tables live in the momentum buffers until Adam state is zeroed below
    dsd = p.m;
    disb = reinterpret_cast<unsigned char*>(p.v);
    cudaMemcpyAsync(dsd, sd.data(), sizeof(float) * n->P, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(disb, isb.data(), n->P, cudaMemcpyHostToDevice, st);
    mrcm::k_init<<<256, 256, 0, st>>>(n->P, p.w, disb, dsd, seed);
    mrcm::k_zero_f<<<256, 256, 0, st>>>(2 * n->P, p.m);
    mrcm::k_to_bf16<<<256, 256, 0, st>>>(n->P, p.w, p.wb);
    cudaError_t e = cudaStreamSynchronize(st);   // host tables must outlive the copies
    return e == cudaSuccess ? MRCM_OK : MRCM_ERR_CUDA;
}

mrcm_status mrcm_net_sync_weights(mrcm_net* n, float* state, void* stream) {
    if (!n || !state) return MRCM_ERR_INVALID_ARG;
    NetPtrs p = net_ptrs(n, state);
    mrcm::k_to_bf16<<<256, 256, 0, (cudaStream_t)stream>>>(n->P, p.w, p.wb);
    return cudaGetLastError() == cudaSuccess ? MRCM_OK : MRCM_ERR_CUDA;
}

mrcm_status mrcm_net_forward(mrcm_net* n, const float* state, const float* x, float* y, int batch, void* ws,
                             void* stream) {
    if (!n || !state || !x || !y || !ws || batch < 1) return MRCM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    NetPtrs p = net_ptrs(n, state);
    float* acts = (float*)ws;
    forward(n, p, x, batch, acts, st);
    cudaMemcpyAsync(y, acts + (long long)batch * n->act_off[n->layers - 1], sizeof(float) * batch * n->S,
                    cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError() == cudaSuccess ? MRCM_OK : MRCM_ERR_CUDA;
}

static float* ws_grad(const mrcm_net* n, void* ws, int batch, float** g0, float** g1, float** partial) {
    float* acts = (float*)ws;
    float* after = acts + (long long)batch * n->act_per_sample;
    *g0 = after;
    *g1 = after + (long long)batch * n->max_ch * n->S;
    *partial = *g1 + (long long)batch * n->max_ch * n->S;
    return *partial + 1024;
}

mrcm_status mrcm_net_gradient(mrcm_net* n, const float* state, const float* x, const float* target,
                              const float* weight, int batch, float* grad, float* loss, void* ws, void* stream) {
    if (!n || !state || !x || !target || !grad || !loss || !ws || batch < 1) return MRCM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    NetPtrs p = net_ptrs(n, state);
    float *g0, *g1, *partial;
    ws_grad(n, ws, batch, &g0, &g1, &partial);
    forward(n, p, x, batch, (float*)ws, st);
    backward(n, p, x, target, weight, batch, (float*)ws, g0, g1, grad, partial, loss, st);
    return cudaGetLastError() == cudaSuccess ? MRCM_OK : MRCM_ERR_CUDA;
}

mrcm_status mrcm_net_train_step(mrcm_net* n, float* state, const float* x, const float* target,
                                const float* weight, int batch, float lr, int step, float* loss, void* ws,
                                void* stream) {
    if (!n || !state || !x || !target || !loss || !ws || batch < 1 || step < 1) return MRCM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    NetPtrs p = net_ptrs(n, state);
    float *g0, *g1, *partial;
    float* grad = ws_grad(n, ws, batch, &g0, &g1, &partial);
    forward(n, p, x, batch, (float*)ws, st);
    backward(n, p, x, target, weight, batch, (float*)ws, g0, g1, grad, partial, loss, st);
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)step), c2 = 1.0f - std::pow(b2, (float)step);
    mrcm::k_adam<<<128, 256, 0, st>>>(n->P, p.w, p.m, p.v, grad, p.wb, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? MRCM_OK : MRCM_ERR_CUDA;
}

void mrcm_net_destroy(mrcm_net* n) { delete n; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Samples and the warm-started local CG, on an MRCM handle after
// mrcm_solve_mbf.  Sample s is the P-MBF column c of subdomain l, for the
// subdomains whose box is W x H x D cells, enumerated by subdomain then c.
// ---------------------------------------------------------------------------
namespace mrcm {
namespace {

__device__ __forceinline__ void slab_coords(const SubInfo& s, int c, int lc[3]) {
    const int sl = c / s.b, r = c - sl * s.b, v = r / s.su;
    lc[s.sa] = sl;
    lc[s.ua] = r - v * s.su;
    lc[s.va] = v;
}

__global__ void __launch_bounds__(256)
k_gather_samples(const SubInfo* __restrict__ subs, const FaceInfo* __restrict__ faces, const int* __restrict__ soff,
                 const double* __restrict__ K, const double* __restrict__ X, int nx, int ny, long long ncells,
                 int max_samples, float* __restrict__ xs, float* __restrict__ ts) {
    const SubInfo s = subs[blockIdx.x];
    const int base = soff[blockIdx.x];
    if (base < 0) return;
    const int N = s.N;
    for (int c = 0; c < s.nI; ++c) {
        const int smp = base + c;
        if (smp >= max_samples) return;
        float* xin = xs + (long long)smp * 4 * N;
        float* tg = ts ? ts + (long long)smp * N : nullptr;
        for (int e = threadIdx.x; e < N; e += blockDim.x) {
            int lc[3];
            slab_coords(s, e, lc);
            const int lex = lc[0] + s.sz[0] * (lc[1] + s.sz[1] * lc[2]);
            const long long gcell = (s.o[0] + lc[0]) + (long long)nx * ((s.o[1] + lc[1]) + (long long)ny * (s.o[2] + lc[2]));
            xin[lex] = kLogKScale * (float)log(K[gcell]);
            xin[N + lex] = kLogKScale * (float)log(K[2 * ncells + gcell]);
            xin[2 * N + lex] = 0.0f;
            xin[3 * N + lex] = 0.0f;
            if (tg) tg[lex] = (float)X[s.x_off + (long long)c * N + e];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < s.nface; q += blockDim.x) {
            const FaceInfo fi = faces[s.face_off + q];
            int lc[3];
            slab_coords(s, fi.cell, lc);
            const int lex = lc[0] + s.sz[0] * (lc[1] + s.sz[1] * lc[2]);
            if (fi.col == c) xin[2 * N + lex] = 1.0f;            // one face per cell for a basis
        }
        __syncthreads();
    }
}

// Robin mask: cells with at least one Robin face (the same for every sample
// of a subdomain), written after the gather for each sample.
__global__ void __launch_bounds__(256)
k_gather_mask(const SubInfo* __restrict__ subs, const FaceInfo* __restrict__ faces, const int* __restrict__ soff,
              int max_samples, float* __restrict__ xs) {
    const SubInfo s = subs[blockIdx.x];
    const int base = soff[blockIdx.x];
    if (base < 0) return;
    const int N = s.N;
    for (int q = threadIdx.x; q < s.nface; q += blockDim.x) {
        const FaceInfo fi = faces[s.face_off + q];
        int lc[3];
        slab_coords(s, fi.cell, lc);
        const int lex = lc[0] + s.sz[0] * (lc[1] + s.sz[1] * lc[2]);
        for (int c = 0; c < s.nI; ++c) {
            const int smp = base + c;
            if (smp < max_samples) xs[(long long)smp * 4 * N + 3 * N + lex] = 1.0f;
        }
    }
}

// Face-flux weights of the loss: per sample and cell, the sum of T_R^2 over
// the cell's Robin faces (zero inside), the same for every sample of a
// subdomain.  One thread per (sample of the subdomain, cell), summing the
// cell's faces in face order (deterministic).
__global__ void __launch_bounds__(256)
k_gather_flux_weights(const SubInfo* __restrict__ subs, const FaceInfo* __restrict__ faces,
                      const double* __restrict__ face_tr, const int* __restrict__ soff, int max_samples,
                      float* __restrict__ wt) {
    const SubInfo s = subs[blockIdx.x];
    const int base = soff[blockIdx.x];
    if (base < 0) return;
    const int N = s.N;
    for (int e = threadIdx.x; e < s.nI * N; e += blockDim.x) {
        const int c = e / N, cell = e - c * N;          // cell in slab order
        if (base + c >= max_samples) continue;
        float acc = 0.0f;
        for (int q = 0; q < s.nface; ++q) {
            const FaceInfo fi = faces[s.face_off + q];
            if (fi.cell != cell) continue;
            const float tr = (float)face_tr[s.face_off + q];
            acc = fmaf(tr, tr, acc);
        }
        int lc[3];
        slab_coords(s, cell, lc);
        wt[(long long)(base + c) * N + lc[0] + s.sz[0] * (lc[1] + s.sz[1] * lc[2])] = acc;
    }
}

// Conjugate gradients in FP32 on the Jacobi-scaled local system A^ = S A S
// (unit diagonal, so Jacobi preconditioning is the identity here) for the
// P-MBF column of one sample, from x0 (unscaled guess, or zero).  The result
// replaces the column of the MBF array (FP64); iterations go to iters[s]
// (maxit + 1 when the tolerance was not reached).
__global__ void __launch_bounds__(512)
k_pcg_sample(const SubInfo* __restrict__ subs, const FaceInfo* __restrict__ faces, const int* __restrict__ slist,
             const double* __restrict__ coef, const double* __restrict__ scale, const double* __restrict__ face_tr,
             long long nct, const float* __restrict__ x0, double* __restrict__ X, int maxit, float tol,
             int* __restrict__ iters) {
    extern __shared__ __align__(16) float sm[];
    const int smp = blockIdx.x;
    const int l = slist[2 * smp], col = slist[2 * smp + 1];
    const SubInfo s = subs[l];
    const int N = s.N, b = s.b, su = s.su;
    float* dd = sm;            // scaled diagonal
    float* tu = dd + N;        // scaled couplings to +u, +v, +slab
    float* tv = tu + N;
    float* ts = tv + N;
    float* x = ts + N;
    float* r = x + N;
    float* p = r + N;
    float* q = p + N;
    __shared__ float red[32];
    const double* cd = coef + s.cell_off;
    const double* cu = coef + nct + s.cell_off;
    const double* cv = coef + 2 * nct + s.cell_off;
    const double* cs = coef + 3 * nct + s.cell_off;
    const double* sc = scale + s.cell_off;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        const int i = c % b, u = i % su;
        dd[c] = (float)(cd[c] * sc[c] * sc[c]);
        tu[c] = u + 1 < su ? (float)(cu[c] * sc[c] * sc[c + 1]) : 0.0f;
        tv[c] = i + su < b ? (float)(cv[c] * sc[c] * sc[c + su]) : 0.0f;
        ts[c] = c + b < N ? (float)(cs[c] * sc[c] * sc[c + b]) : 0.0f;
        r[c] = 0.0f;
        float xv = 0.0f;
        if (x0) {
            int lc[3];
            slab_coords(s, c, lc);
            const int lex = lc[0] + s.sz[0] * (lc[1] + s.sz[1] * lc[2]);
            xv = (float)(x0[(long long)smp * N + lex] / sc[c]);
        }
        x[c] = xv;
    }
    __syncthreads();
    for (int f = threadIdx.x; f < s.nface; f += blockDim.x) {
        const FaceInfo fi = faces[s.face_off + f];
        if (fi.col == col) r[fi.cell] = (float)(face_tr[s.face_off + f] * sc[fi.cell]);   // b^ = S b
    }
    __syncthreads();
    auto matvec = [&](const float* v, float* out) {
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
            const int i = c % b, u = i % su;
            float a = dd[c] * v[c];
            if (u + 1 < su) a -= tu[c] * v[c + 1];
            if (u > 0) a -= tu[c - 1] * v[c - 1];
            if (i + su < b) a -= tv[c] * v[c + su];
            if (i >= su) a -= tv[c - su] * v[c - su];
            if (c + b < N) a -= ts[c] * v[c + b];
            if (c >= b) a -= ts[c - b] * v[c - b];
            out[c] = a;
        }
    };
    auto dot = [&](const float* a, const float* bb) -> float {
        float acc = 0.0f;
        for (int c = threadIdx.x; c < N; c += blockDim.x) acc = fmaf(a[c], bb[c], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        return t;
    };
    const float bnorm2 = dot(r, r);
    matvec(x, q);
    __syncthreads();
    for (int c = threadIdx.x; c < N; c += blockDim.x) { r[c] -= q[c]; p[c] = r[c]; }
    __syncthreads();
    float rr = dot(r, r);
    int it = 0;
    const float tol2 = tol * tol * bnorm2;
    while (rr > tol2 && it < maxit) {
        matvec(p, q);
        __syncthreads();
        const float pq = dot(p, q);
        const float alpha = rr / pq;
        for (int c = threadIdx.x; c < N; c += blockDim.x) { x[c] += alpha * p[c]; r[c] -= alpha * q[c]; }
        __syncthreads();
        const float rr2 = dot(r, r);
        const float beta = rr2 / rr;
        rr = rr2;
        for (int c = threadIdx.x; c < N; c += blockDim.x) p[c] = r[c] + beta * p[c];
        __syncthreads();
        ++it;
    }
    for (int c = threadIdx.x; c < N; c += blockDim.x) X[s.x_off + (long long)col * N + c] = (double)x[c] * sc[c];
    if (threadIdx.x == 0) iters[smp] = rr > tol2 ? maxit + 1 : it;
}

// Learned form of the local solves (one CTA per MBF or particular column):
// FP64 iterative refinement, r = b - A x in FP64, whose correction equations
// A^ z = S r are solved by FP32 conjugate gradients on the Jacobi-scaled
// system to a relative residual of 1e-4 (or cg_maxit iterations), x += S z.
// The start x0 is the network's prediction for a P-MBF column, -beta s times
// that prediction for the U-MBF column of the same basis (exact when beta is
// constant on the patch), zero for the particular column.  A column whose
// FP64 residual reaches ||r|| <= tol ||b|| gets conv = 1; the others are left
// to the FP64 direct fallback.
__device__ __forceinline__ double block_sum_d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

__global__ void __launch_bounds__(256)
k_learned_column(const SubInfo* __restrict__ subs, const FaceInfo* __restrict__ faces, const int* __restrict__ col_list,
                 const double* __restrict__ coef, const double* __restrict__ scale,
                 const double* __restrict__ face_tr, const double* __restrict__ face_u,
                 const double* __restrict__ face_beta, const double* __restrict__ rhs_part,
                 const double* __restrict__ f, int nx, int ny, double vol, long long nct,
                 const int* __restrict__ soff, const float* __restrict__ pred, int n_pred, int cg_maxit,
                 int max_outer, double tol, double* __restrict__ X, int* __restrict__ conv, int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char lsm[];
    const int l = col_list[2 * blockIdx.x], j = col_list[2 * blockIdx.x + 1];
    const SubInfo s = subs[l];
    const int N = s.N, b = s.b, su = s.su, nI = s.nI, m = s.m;
    double* x = reinterpret_cast<double*>(lsm);
    double* bb = x + N;
    float* dd = reinterpret_cast<float*>(bb + N);
    float* tu = dd + N;
    float* tv = tu + N;
    float* ts = tv + N;
    float* z = ts + N;
    float* r = z + N;
    float* p = r + N;
    float* q = p + N;
    __shared__ float red[32];
    __shared__ double redd[32];
    __shared__ double wscale_s;
    const double* cd = coef + s.cell_off;
    const double* cu = coef + nct + s.cell_off;
    const double* cv = coef + 2 * nct + s.cell_off;
    const double* cs = coef + 3 * nct + s.cell_off;
    const double* sc = scale + s.cell_off;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        const int i = c % b, u = i % su;
        dd[c] = (float)(cd[c] * sc[c] * sc[c]);
        tu[c] = u + 1 < su ? (float)(cu[c] * sc[c] * sc[c + 1]) : 0.0f;
        tv[c] = i + su < b ? (float)(cv[c] * sc[c] * sc[c + su]) : 0.0f;
        ts[c] = c + b < N ? (float)(cs[c] * sc[c] * sc[c + b]) : 0.0f;
        double bv = 0.0;
        if (j == m - 1) {
            int lc[3];
            slab_coords(s, c, lc);
            const long long g = (s.o[0] + lc[0]) + (long long)nx * ((s.o[1] + lc[1]) + (long long)ny * (s.o[2] + lc[2]));
            bv = rhs_part[s.cell_off + c] + f[g] * vol;
        }
        bb[c] = bv;
        x[c] = 0.0;
    }
    if (threadIdx.x == 0) wscale_s = 1.0;
    __syncthreads();
    const int pc = j < nI ? j : (j < 2 * nI ? j - nI : -1);       // the basis of an MBF column
    if (j < m - 1) {
        for (int e = threadIdx.x; e < s.nface; e += blockDim.x) {
            const FaceInfo fi = faces[s.face_off + e];
            if (fi.col != pc) continue;
            bb[fi.cell] = j < nI ? face_tr[s.face_off + e] : face_u[s.face_off + e];
            if (j >= nI) wscale_s = -face_beta[s.face_off + e] * fi.s;    // any face of the basis (a benign race)
        }
    }
    __syncthreads();
    if (pred && soff && pc >= 0 && soff[l] >= 0 && soff[l] + pc < n_pred) {
        const float* pr = pred + (long long)(soff[l] + pc) * N;
        const double ws = j < nI ? 1.0 : wscale_s;
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
            int lc[3];
            slab_coords(s, c, lc);
            x[c] = ws * (double)pr[lc[0] + s.sz[0] * (lc[1] + s.sz[1] * lc[2])];
        }
    }
    __syncthreads();
    auto matvec = [&](const float* v, float* out) {
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
            const int i = c % b, u = i % su;
            float a = dd[c] * v[c];
            if (u + 1 < su) a -= tu[c] * v[c + 1];
            if (u > 0) a -= tu[c - 1] * v[c - 1];
            if (i + su < b) a -= tv[c] * v[c + su];
            if (i >= su) a -= tv[c - su] * v[c - su];
            if (c + b < N) a -= ts[c] * v[c + b];
            if (c >= b) a -= ts[c - b] * v[c - b];
            out[c] = a;
        }
    };
    auto dot = [&](const float* a, const float* bv) -> float {
        float acc = 0.0f;
        for (int c = threadIdx.x; c < N; c += blockDim.x) acc = fmaf(a[c], bv[c], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        return t;
    };
    double bn = 0.0;
    for (int c = threadIdx.x; c < N; c += blockDim.x) bn += bb[c] * bb[c];
    bn = block_sum_d(bn, redd);
    long long iters = 0;
    int ok = 0;
    for (int o = 0; o <= max_outer; ++o) {
        // FP64 residual of the unscaled system, the scaled right-hand side of the correction
        double rr = 0.0;
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
            const int i = c % b, u = i % su;
            double a = cd[c] * x[c];
            if (u + 1 < su) a = fma(-cu[c], x[c + 1], a);
            if (u > 0) a = fma(-cu[c - 1], x[c - 1], a);
            if (i + su < b) a = fma(-cv[c], x[c + su], a);
            if (i >= su) a = fma(-cv[c - su], x[c - su], a);
            if (c + b < N) a = fma(-cs[c], x[c + b], a);
            if (c >= b) a = fma(-cs[c - b], x[c - b], a);
            const double res = bb[c] - a;
            rr = fma(res, res, rr);
            r[c] = (float)(res * sc[c]);
            z[c] = 0.0f;
            p[c] = r[c];
        }
        rr = block_sum_d(rr, redd);
        if (rr <= tol * tol * bn) { ok = 1; break; }
        if (o == max_outer) break;
        float rho = dot(r, r);
        const float stop = 1e-8f * rho;                  // relative residual 1e-4
        for (int k = 0; k < cg_maxit && rho > stop; ++k) {
            matvec(p, q);
            __syncthreads();
            const float alpha = rho / dot(p, q);
            for (int c = threadIdx.x; c < N; c += blockDim.x) { z[c] = fmaf(alpha, p[c], z[c]); r[c] = fmaf(-alpha, q[c], r[c]); }
            __syncthreads();
            const float rho2 = dot(r, r);
            const float beta = rho2 / rho;
            rho = rho2;
            for (int c = threadIdx.x; c < N; c += blockDim.x) p[c] = fmaf(beta, p[c], r[c]);
            __syncthreads();
            ++iters;
        }
        for (int c = threadIdx.x; c < N; c += blockDim.x) x[c] = fma((double)z[c], sc[c], x[c]);
        __syncthreads();
    }
    double* Xc = X + s.x_off + (long long)j * N;
    for (int c = threadIdx.x; c < N; c += blockDim.x) Xc[c] = x[c];
    if (threadIdx.x == 0) {
        conv[s.rhs_off + j] = ok;
        atomicAdd(reinterpret_cast<unsigned long long*>(status + ST_CG_ITERS), (unsigned long long)iters);
    }
}

}  // namespace
}  // namespace mrcm

namespace {

// Sample enumeration of a handle for a box shape: per-subdomain first sample
// (or -1) and the (subdomain, column) list; an internal table of the handle.
mrcm_status sample_tables(mrcm_handle* h, int D, int H, int W, int** soff_d, int** slist_d, int* count) {
    const mrcm::Tables& t = h->t;
    if (h->samp_shape[0] == D && h->samp_shape[1] == H && h->samp_shape[2] == W && h->samp_off) {
        *soff_d = h->samp_off;
        *slist_d = h->samp_list;
        *count = h->samp_count;
        return MRCM_OK;
    }
    if (h->samp_off) cudaFree(h->samp_off);
    if (h->samp_list) cudaFree(h->samp_list);
    h->samp_off = h->samp_list = nullptr;
    std::vector<int> off(t.subs.size(), -1), lst;
    int n = 0;
    for (size_t l = 0; l < t.subs.size(); ++l) {
        const mrcm::SubInfo& s = t.subs[l];
        if (s.sz[0] != W || s.sz[1] != H || s.sz[2] != D) continue;
        off[l] = n;
        for (int c = 0; c < s.nI; ++c) { lst.push_back((int)l); lst.push_back(c); }
        n += s.nI;
    }
    if (cudaMalloc((void**)&h->samp_off, sizeof(int) * std::max<size_t>(off.size(), 1)) != cudaSuccess ||
        cudaMalloc((void**)&h->samp_list, sizeof(int) * std::max<size_t>(lst.size(), 1)) != cudaSuccess)
        return MRCM_ERR_CUDA;
    cudaMemcpy(h->samp_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice);
    if (!lst.empty()) cudaMemcpy(h->samp_list, lst.data(), sizeof(int) * lst.size(), cudaMemcpyHostToDevice);
    h->samp_shape[0] = D; h->samp_shape[1] = H; h->samp_shape[2] = W;
    h->samp_count = n;
    *soff_d = h->samp_off;
    *slist_d = h->samp_list;
    *count = n;
    return MRCM_OK;
}

}  // namespace

extern "C" {

mrcm_status mrcm_net_samples(mrcm_handle* h, const mrcm_net* net, void* ws, float* x, float* target,
                             int max_samples, int* n_samples, void* stream) {
    if (!h || !net || !ws || !n_samples) return MRCM_ERR_INVALID_ARG;
    if (h->stage < (target ? 2 : 1)) return MRCM_ERR_STATE;     // inputs need K, targets the MBFs
    if (net->in_ch != 4) return MRCM_ERR_INVALID_ARG;
    int *soff, *slist, cnt;
    mrcm_status st = sample_tables(h, net->D, net->H, net->W, &soff, &slist, &cnt);
    if (st != MRCM_OK) return st;
    *n_samples = std::min(cnt, std::max(max_samples, 0));
    if (!x || *n_samples == 0) return MRCM_OK;
    const mrcm::Tables& t = h->t;
    cudaStream_t s = (cudaStream_t)stream;
    mrcm::k_gather_samples<<<(int)t.subs.size(), 256, 0, s>>>(h->d.subs, h->d.faces, soff, h->K,
        (const double*)((char*)ws + h->lay.X), t.cfg.nx, t.cfg.ny, t.n_cells, max_samples, x, target);
    mrcm::k_gather_mask<<<(int)t.subs.size(), 256, 0, s>>>(h->d.subs, h->d.faces, soff, max_samples, x);
    return cudaGetLastError() == cudaSuccess ? MRCM_OK : MRCM_ERR_CUDA;
}

mrcm_status mrcm_net_flux_weights(mrcm_handle* h, const mrcm_net* net, void* ws, float* weight, int max_samples,
                                  void* stream) {
    if (!h || !net || !ws || !weight || max_samples < 0) return MRCM_ERR_INVALID_ARG;
    if (h->stage < 1) return MRCM_ERR_STATE;
    int *soff, *slist, cnt;
    mrcm_status st = sample_tables(h, net->D, net->H, net->W, &soff, &slist, &cnt);
    if (st != MRCM_OK) return st;
    if (max_samples == 0) return MRCM_OK;
    mrcm::k_gather_flux_weights<<<(int)h->t.subs.size(), 256, 0, (cudaStream_t)stream>>>(h->d.subs, h->d.faces,
        (const double*)((char*)ws + h->lay.face_tr), soff, std::min(max_samples, cnt), weight);
    return cudaGetLastError() == cudaSuccess ? MRCM_OK : MRCM_ERR_CUDA;
}

mrcm_status mrcm_solve_mbf_learned(mrcm_handle* h, const mrcm_net* net, const float* pred, int n_pred,
                                   const double* f, int cg_maxit, int max_outer, void* ws, void* stream) {
    if (!h || !ws || !f || cg_maxit < 0 || max_outer < 0 || n_pred < 0) return MRCM_ERR_INVALID_ARG;
    const mrcm::Tables& t = h->t;
    if (t.cfg.precision != MRCM_LEARNED_PCG) { h->err = "handle precision is not MRCM_LEARNED_PCG"; return MRCM_ERR_INVALID_ARG; }
    if (h->stage < 1) { h->err = "mrcm_factor_local must run first"; return MRCM_ERR_STATE; }
    if (pred && (!net || net->in_ch != 4)) return MRCM_ERR_INVALID_ARG;
    if (t.max_N > 4096) return MRCM_ERR_NOT_IMPLEMENTED;
    if (!h->col_list) {
        std::vector<int> cl;
        for (size_t l = 0; l < t.subs.size(); ++l)
            for (int j = 0; j < t.subs[l].m; ++j) { cl.push_back((int)l); cl.push_back(j); }
        if (cudaMalloc((void**)&h->col_list, sizeof(int) * std::max<size_t>(cl.size(), 1)) != cudaSuccess)
            return MRCM_ERR_CUDA;
        cudaMemcpy(h->col_list, cl.data(), sizeof(int) * cl.size(), cudaMemcpyHostToDevice);
        h->n_cols = (int)(cl.size() / 2);
    }
    int* soff = nullptr;
    if (pred) {
        int *slist, cnt;
        mrcm_status st = sample_tables(h, net->D, net->H, net->W, &soff, &slist, &cnt);
        if (st != MRCM_OK) return st;
        n_pred = std::min(n_pred, cnt);
    }
    h->f = f;
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)ws;
    int* status = (int*)(w + h->lay.status);
    cudaMemsetAsync(status, 0, sizeof(int) * mrcm::ST_COUNT, st);
    const size_t sm = (size_t)t.max_N * (2 * sizeof(double) + 8 * sizeof(float));
    cudaFuncSetAttribute(mrcm::k_learned_column, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const double tol = t.cfg.ir_tol > 0 ? t.cfg.ir_tol : 1e-9;
    if (h->n_cols > 0)
        mrcm::k_learned_column<<<h->n_cols, 256, sm, st>>>(h->d.subs, h->d.faces, h->col_list,
            (const double*)(w + h->lay.coef), (const double*)(w + h->lay.scale), (const double*)(w + h->lay.face_tr),
            (const double*)(w + h->lay.face_u), (const double*)(w + h->lay.face_beta),
            (const double*)(w + h->lay.rhs_part), f, t.cfg.nx, t.cfg.ny, t.cfg.hx * t.cfg.hy * t.cfg.hz, t.n_cells,
            soff, pred, n_pred, cg_maxit, max_outer, tol, (double*)(w + h->lay.X), (int*)(w + h->lay.conv), status);
    int rc = mrcm::launch_local_finish(t, h->d, h->lay, w, f, stream, h->prof);
    if (rc != 0 || cudaGetLastError() != cudaSuccess) { h->err = "mrcm_solve_mbf_learned: launch failed"; return MRCM_ERR_CUDA; }
    h->stage = 2;
    return MRCM_OK;
}

mrcm_status mrcm_read_cg_iterations(mrcm_handle* h, void* ws, long long* iters) {
    if (!h || !ws || !iters) return MRCM_ERR_INVALID_ARG;
    unsigned long long v = 0;
    if (cudaMemcpy(&v, (char*)ws + h->lay.status + mrcm::ST_CG_ITERS * sizeof(int), sizeof(v),
                   cudaMemcpyDeviceToHost) != cudaSuccess) return MRCM_ERR_CUDA;
    *iters = (long long)v;
    return MRCM_OK;
}

mrcm_status mrcm_pcg_mbf(mrcm_handle* h, const mrcm_net* net, void* ws, const float* x0, int n_samples,
                         int maxit, double tol, int* iters, void* stream) {
    if (!h || !net || !ws || !iters || maxit < 0 || !(tol > 0)) return MRCM_ERR_INVALID_ARG;
    if (h->stage < 1) return MRCM_ERR_STATE;
    int *soff, *slist, cnt;
    mrcm_status st = sample_tables(h, net->D, net->H, net->W, &soff, &slist, &cnt);
    if (st != MRCM_OK) return st;
    if (n_samples < 0 || n_samples > cnt) return MRCM_ERR_INVALID_ARG;
    if (n_samples == 0) return MRCM_OK;
    const mrcm::Tables& t = h->t;
    if (net->S > 1024) return MRCM_ERR_NOT_IMPLEMENTED;
    const size_t sm = sizeof(float) * 8 * (size_t)net->S;
    cudaFuncSetAttribute(mrcm::k_pcg_sample, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const char* w = (const char*)ws;
    mrcm::k_pcg_sample<<<n_samples, 512, sm, (cudaStream_t)stream>>>(h->d.subs, h->d.faces, slist,
        (const double*)(w + h->lay.coef), (const double*)(w + h->lay.scale), (const double*)(w + h->lay.face_tr),
        t.n_cells, x0, (double*)(w + h->lay.X), maxit, (float)tol, iters);
    return cudaGetLastError() == cudaSuccess ? MRCM_OK : MRCM_ERR_CUDA;
}

}  // extern "C"
