// Internal tables shared by the host setup and the CUDA kernels of libmrcm.
#pragma once
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mrcm.h"
#include "mrcm_prof.h"

namespace mrcm {

constexpr int kMaxBlock = 256;      // largest slab block b (FP32 factor; FP64 factor: kMaxBlock64)
constexpr int kMaxBlock64 = 224;    // largest slab block b whose FP64 packed triangle fits shared memory (larger: global slot)
constexpr int kRegBlock = 64;       // blocks with b <= kRegBlock use the register-resident FP32 factor
constexpr int kMaxSolveVariants = 16;  // capacity of the per-variant tables
constexpr int kNumFactorVariants = 3;  // factor kernels for blocks with b <= 64
constexpr int kOzMinN = 32;        // fronts with n >= kOzMinN may take the tensor-core emulated FP64 update
constexpr int kOzMinM = 24;        // a step emulates when the trailing block has >= kOzMinM rows
constexpr int kOzMinK = 4;         // and the panel >= kOzMinK columns
// BF16 flops one 32 x 32 tile of the emulated update executes: 8 warps x 36 slice pairs
// (8 slices per operand, pairs with t + u < 8) x 2 halves of the panel x m16n8k16 MMAs
constexpr double kOzTileFlops = 8.0 * 36.0 * 2.0 * (2.0 * 16 * 8 * 16);
constexpr int kTileBlock = 128;     // 64 < b <= kTileBlock: register-tiled FP32 factor (8 x 8 per thread)
constexpr int kMaxI = 128;          // largest |I^l| (basis functions touching one subdomain)

// One subdomain.  Local cells are numbered slab-major: the slab axis `sa` is
// the subdomain's longest axis; inside a slab the two other axes (ua < va)
// run u fastest.  local = s*b + u + su*v.  With this order the local TPFA
// matrix is block tridiagonal with b x b diagonal blocks (5-point stencils)
// and diagonal coupling blocks between consecutive slabs.
struct SubInfo {
    int o[3];          // origin (cells)
    int sz[3];         // extents
    int sa, ua, va;    // slab axis, fast and slow in-slab axes
    int su, sv, b, ns, N;
    int nI;            // |I^l|
    int m;             // 2|I^l| + 1 right-hand sides
    int face_off, nface;
    int I_off;         // offset into the I^l lists
    int el_dim;        // 2|I^l|
    long long cell_off;   // offset into per-cell arrays
    long long x_off;      // offset (doubles) into the MBF array [m][N]
    long long y_off;      // offset (elements) of the forward-sweep values Y (= x_off; a slot for the FP64 fallback)
    int big_slot;         // FP64 form, b > kMaxBlock64: the subdomain's slot (in its wave) of the factor's
                          // packed triangle in global memory; -1 = the triangle fits shared memory
    long long w_off;      // offset (elements) into the block factor array
    long long el_off;     // offset (doubles) into element matrices
    int elb_off;          // offset (doubles) into element right-hand sides
    int rhs_off;          // offset of the subdomain's columns in per-column arrays
};

// One Robin face of a subdomain (a fine face of Gamma seen from one side).
struct FaceInfo {
    int cell;          // local cell (slab order)
    int col;           // position of its basis in I^l
    int8_t axis;       // normal axis
    int8_t s;          // +1 lower side, -1 upper side
    int16_t pad;
};

// One internal node of the interface elimination tree (a dense front).
struct FrontInfo {
    int ne, nb, n;          // eliminated dofs, boundary dofs, n = ne + nb
    int nchild;             // 2
    long long f_off;        // offset (doubles) of the n x n front (row major)
    int r_off;              // offset (doubles) of the front right-hand side
    int child[2];           // child front index, or -(1 + element) for a leaf
    int map_off[2];         // offset (ints) of the child -> front position maps
    int map_len[2];
    int inv_off;            // offset (ints) of the front -> child position maps (2 x n, -1 = absent)
    int e_dof_off;          // offset (ints) into the global dof list of E then B
    int pin_row;            // front row of pi^p_0 when it is regularised, or -1
    int p_off;              // first of its ceil(ne / 32) inverse diagonal blocks (32 x 32 each)
    int s_off;              // first row of its slice rows in the emulated-update buffer, or -1
    int height;
    int parent;
};

struct Tables {
    // configuration
    mrcm_config cfg;
    std::string tune_cache;
    std::vector<int> cuts[3];
    int N[3];                      // subdomains per axis
    std::vector<int> starts[3];
    bool has_dirichlet = false;

    // subdomains and faces
    std::vector<SubInfo> subs;
    std::vector<FaceInfo> faces;
    std::vector<int> Ilist;        // concatenated sorted I^l (global basis ids)
    std::vector<int> class_list;   // subdomains grouped by factor class, costliest first
    std::vector<int> solve_list;   // all subdomains, costliest solve first
    // memory-bounded waves (cfg.wave_bytes): wave w owns solve_list entries
    // [wave_off[w], wave_off[w+1]); its factor classes are wave_class[w][0..1]
    // (offsets into class_list); block factors are stored per wave (w_off is
    // relative to the wave) so one W region serves every wave
    std::vector<int> wave_off;
    std::vector<int> wave_class_off;   // 4 entries per wave (class boundaries)
    int n_waves = 1;
    int class_off[4] = {0, 0, 0, 0};  // class 0: b <= kRegBlock, 1: b <= kTileBlock, 2: larger (mixed); FP64: all in 2
    long long n_cells = 0, total_x = 0, total_w = 0, total_el = 0;
    int total_elb = 0;
    int max_m = 0, max_b = 0, max_el = 0, max_N = 0;
    long long total_rhs = 0;

    // bases
    int NV = 0;
    std::vector<int> b_axis, b_lo, b_hi, b_nfaces;

    // interface CSR with two-sided sources (element entry offsets or -1)
    std::vector<int> rowptr, colidx;
    std::vector<long long> src_lo, src_hi;
    std::vector<int> rhs_src_lo, rhs_src_hi;   // element rhs offsets per global dof

    // elimination tree
    std::vector<FrontInfo> fronts;
    std::vector<int> front_maps;               // child -> front position maps
    std::vector<int> front_inv;                // front -> child position maps
    std::vector<int> front_dofs;               // global dof of each front row
    std::vector<std::vector<int>> levels;      // fronts grouped by height
    long long total_front = 0;
    int total_frhs = 0;
    int total_panels = 0;          // sum over fronts of ceil(ne / 32)
    long long oz_rows = 0;         // slice rows of the emulated trailing update (max over levels)
    int max_front = 0;
    double front_flops = 0, ldl_flops = 0, ldl_update_flops = 0, ldl_update_tensor_flops = 0, local_factor_flops = 0, local_solve_flops = 0;
    int root = -1;
    int pin_front = -1;

    // mixed modes: the FP64 post-processing factors the Neumann problems into
    // the W region in FP64 waves (pp_wave_off into solve_list; pp_subs are the
    // subdomain records with the FP64 block offsets and one forward-value
    // column per cell); pp_ok is false when some block cannot take it
    std::vector<SubInfo> pp_subs;
    std::vector<int> pp_wave_off;
    bool pp_ok = true;
    int big_slots = 0;             // FP64 form: most subdomains of one wave with b > kMaxBlock64
};

// Workspace layout (byte offsets into the caller's workspace).
struct Layout {
    size_t coef, scale, scf, tsc, rhs_part, face_tr, face_beta, face_u, face_bst, W, X, R, colnorm, conv;
    size_t elem, elem_b, csr_val, b_int, dscale, fronts, frhs, panel, oz, oz_exp, xres, xtmp, psum, status;
    size_t bpart, bcnt;    // row-chunk partial sums and counters of the split boundary back substitution
    size_t fb_W, fb_Y, fb_subs, fb_list;   // FP64 fallback: block factors, forward values, subdomain records, slots
    size_t pp_list;                        // post-processing (mixed): the subdomains its FP32 pass left unconverged
    size_t big;                            // FP64 form: packed triangles of blocks with b > kMaxBlock64 (one wave)
    size_t total;
};

struct DeviceTables {
    SubInfo* subs = nullptr;
    FaceInfo* faces = nullptr;
    int* Ilist = nullptr;
    int* class_list = nullptr;
    int class_off[4] = {0, 0, 0, 0};
    int* solve_list = nullptr;                 // all subdomains, costliest solve first (wave by wave)
    int sms = 0;
    size_t solve_smem = 0;
    int factor_variant = 1;                    // blocks with b <= 64: 0 row per thread, 1 8x8 tiles, 2 4x4 tiles
    int factor_mid_variant = 0;                // 64 < b <= 128: 0 register tiles, 1 tensor cores (TMEM)
    int solve_occ[kMaxSolveVariants] = {};
    int sweep_occ[kMaxSolveVariants] = {};
    int solve_variant = 0, sweep_variant = 0;  // chosen by the autotuner (or the tune cache)
    int sweeps_separate = 0;                   // 1: one launch per refinement sweep, 0: all sweeps in one
                                               // launch (autotuner or tune cache; default 0)
    float sweeps_separate_ms = -1.0f;          // last autotune: the chosen sweep variant, one launch per sweep
    size_t front_smem = 0;
    int* rowptr = nullptr;
    int* colidx = nullptr;
    long long* src_lo = nullptr;
    long long* src_hi = nullptr;
    int* rhs_src_lo = nullptr;
    int* rhs_src_hi = nullptr;
    FrontInfo* fronts = nullptr;
    int* front_maps = nullptr;
    int* front_inv = nullptr;
    int* front_dofs = nullptr;
    int* level_ids = nullptr;                  // fronts of all levels, concatenated
    size_t f64_solve_smem = 0;                 // mixed modes: dynamic shared memory of the FP64 solve kernels
    int f64_occ = 1;                           // (fallback, post-processing) and their CTAs per SM
    SubInfo* pp_subs = nullptr;
    std::vector<int> level_off;                // host: offsets of each level in level_ids
    int device = -1;
    bool ready = false;
};

// Shared-memory layout of k_local_solve: Z and Yp (b x mpad of T each, so
// the column blocks stay 16-byte aligned for vector loads), column norms,
// active columns, the per-cell Robin-face map (six sides per cell) and, for
// blocks with b <= kSmemW, the staged block W_s (larger blocks are read from
// global memory, where they stay L2-resident for the slab).
// Slab block W_s storage: b x b entries padded to a multiple of 16 bytes, so
// that every block starts 16-byte aligned (bulk-copy rule).
template <typename T>
#ifdef __CUDACC__
__host__ __device__
#endif
inline long long wstride(int b) {
    const long long q = 16 / (long long)sizeof(T);
    return ((long long)b * b + q - 1) / q * q;
}

// Shared memory of the local solve for one subdomain.  W blocks are staged by
// bulk copies into nbuf buffers (2: the next block streams in while the
// current one is used; 1 when two would not leave room for two CTAs per SM;
// 0: too large to stage, read from global memory).
constexpr size_t kSolveSmemBudget = 220 * 1024;   // dynamic shared memory per CTA
constexpr size_t kSolveTwoCta = 113 * 1024;       // two CTAs per SM fit below this

struct SolveSmem {
    size_t w, z, yp, nrm, cols, cf, co, total;
    int nbuf;
};

template <typename T>
#ifdef __CUDACC__
__host__ __device__
#endif
inline SolveSmem solve_smem_layout(int b, int mpad, int N) {
    SolveSmem L;
    const size_t wb = sizeof(T) * (size_t)wstride<T>(b);
    size_t rest = 0;
    rest += 2 * sizeof(T) * (size_t)b * mpad;              // Z, Yp
    rest = (rest + 15) & ~size_t(15);
    rest += sizeof(double) * mpad + sizeof(int) * mpad;    // nrm, cols
    rest += sizeof(short) * 6 * (size_t)N;                 // cf
    rest = (rest + 15) & ~size_t(15);
    rest += (5 * sizeof(double) + sizeof(float) + sizeof(T) + sizeof(unsigned) + 6) * (size_t)b + 16;
                                                      // one slab's stencil coefficients, scale, slab
                                                      // coupling, cell masks and face columns
    rest += 16;                                            // mbarriers (after the largest layout)
    L.nbuf = (2 * wb + rest + 128 <= kSolveTwoCta) ? 2 : (wb + rest + 128 <= kSolveSmemBudget ? 1 : 0);
    size_t x = 0;
    L.w = 0;
    x += L.nbuf * ((wb + 127) & ~size_t(127));
    L.z = x;
    x += sizeof(T) * (size_t)b * mpad;
    L.yp = x;
    x += sizeof(T) * (size_t)b * mpad;
    x = (x + 15) & ~size_t(15);
    L.nrm = x;
    x += sizeof(double) * mpad;
    L.cols = x;
    x += sizeof(int) * mpad;
    L.cf = x;
    x += sizeof(short) * 6 * (size_t)N;
    x = (x + 15) & ~size_t(15);
    L.co = x;
    x += (5 * sizeof(double) + sizeof(float) + sizeof(T) + sizeof(unsigned) + 6) * (size_t)b + 16;
    L.total = (x + 127) & ~size_t(127);
    return L;
}

// Row chunks of the boundary back substitution for a level whose fronts have
// at most max_nb boundary rows (about 128 rows per chunk, at most 8 chunks).
inline int bwd_split(int max_nb) { return std::max(1, std::min(8, (max_nb + 127) / 128)); }

// Sizes (doubles, counters) of the split back substitution's work arrays: the
// largest level's (fronts x column blocks x chunks x 32) and (fronts x column blocks).
inline void bwd_split_sizes(const std::vector<std::vector<int>>& levels, const std::vector<FrontInfo>& fronts,
                            size_t* parts, size_t* counters) {
    *parts = 32;
    *counters = 1;
    for (const auto& lv : levels) {
        int mne = 0, mnb = 0;
        for (int id : lv) { mne = std::max(mne, fronts[id].ne); mnb = std::max(mnb, fronts[id].nb); }
        const size_t slots = lv.size() * (size_t)std::max(1, (mne + 31) / 32);
        *parts = std::max(*parts, slots * bwd_split(mnb) * 32);
        *counters = std::max(*counters, slots);
    }
}

// Device status words at Layout::status.
enum StatusWord { ST_NOT_SPD = 0, ST_UNCONVERGED = 1, ST_ZERO_PIVOT = 2, ST_SWEEPS = 3,
                  ST_TIMEOUT = 4, ST_QUEUE = 5 /* work-queue counter */,
                  ST_FB_WAVE = 6 /* fallback slots taken in the current wave */,
                  ST_FB_TOTAL = 7 /* subdomains re-solved in FP64 */,
                  ST_SWEPT = 8 /* 64-bit counter at words 8-9 */,
                  ST_FB_LOST = 10 /* subdomains that needed the fallback and could not have it */,
                  ST_CG_ITERS = 12 /* 64-bit counter at words 12-13: CG iterations of the learned form */,
                  ST_COUNT = 16 };

// FP64 fallback of the mixed modes: slots per wave and FP64 block-factor
// doubles per slot (the largest n_s x padded b^2 among blocks the FP64 factor
// takes, b <= kMaxBlock64); cap 0 = no fallback.
inline void fallback_params(const Tables& t, int* cap, long long* stride, long long* ystride = nullptr) {
    *cap = 0;
    *stride = 0;
    if (ystride) *ystride = 0;
    const int nsub = (int)t.subs.size();
    if (t.cfg.precision == MRCM_FP64 || t.cfg.fallback_cap < 0 || nsub == 0) return;
    long long st = 0, yst = 0;
    for (const SubInfo& s : t.subs)
        if (s.b <= kMaxBlock64) {
            st = std::max(st, (long long)s.ns * wstride<double>(s.b));
            yst = std::max(yst, (long long)s.m * s.N);
        }
    if (st == 0) return;
    *stride = (st + 31) / 32 * 32;
    if (ystride) *ystride = (yst + 31) / 32 * 32;
    *cap = t.cfg.fallback_cap > 0 ? std::min(t.cfg.fallback_cap, nsub) : std::min(nsub, std::max(16, nsub / 64));
}

}  // namespace mrcm

struct mrcm_handle {
    mrcm::Tables t;
    mrcm::Layout lay;
    mrcm::DeviceTables d;
    mrcm::Prof prof;
    std::string err;
    int stage = 0;     // 0 setup, 1 factored, 2 mbf, 3 assembled, 4 interface solved
    cudaGraph_t graph = nullptr;          // captured solve (mrcm_solve with MRCM_SOLVE_GRAPH)
    cudaGraphExec_t graph_exec = nullptr;
    const void* graph_key[9] = {};
    long long graph_launches = 0;
    // host-buffer solve (mrcm_solve_host): device staging, a side stream for parallel copies, its graph
    double* io = nullptr;
    size_t io_bytes = 0;
    cudaStream_t io_side = nullptr;
    cudaEvent_t io_ev[2] = {nullptr, nullptr};
    cudaGraph_t hgraph = nullptr;
    cudaGraphExec_t hgraph_exec = nullptr;
    const void* hgraph_key[10] = {};
    long long hgraph_launches = 0;
    float tune_ms[2 * mrcm::kMaxSolveVariants] = {};   // last autotune: first solve / sweeps per variant
    int tune_n = 0;                                    // variants timed (0: no autotune yet)
    int* col_list = nullptr;              // learned-path (subdomain, column) list of every MBF column
    int n_cols = 0;
    int* samp_off = nullptr;              // learned-path sample tables (internal)
    int* samp_list = nullptr;
    int samp_shape[3] = {0, 0, 0};
    int samp_count = 0;
    const double* K = nullptr;   // caller's K (kept for reconstruction)
    const double* f = nullptr;   // caller's f
};

// Host setup (mrcm_setup.cpp)
namespace mrcm {
mrcm_status build_tables(const mrcm_config* cfg, Tables& t, std::string& err);
void min_degree_cost(int sx, int sy, int sz, double* flops, long long* nnz);
void compute_layout(const Tables& t, Layout& lay);
}

// Kernel launchers (CUDA translation units).  Each returns cudaError_t as int.
namespace mrcm {
int num_solve_variants();
int launch_factor(const Tables& t, const DeviceTables& d, const Layout& L, char* ws,
                  const double* K, int precision, void* stream, Prof& P);
int launch_solve_mbf(const Tables& t, const DeviceTables& d, const Layout& L, char* ws,
                     const double* f, int precision, int sweeps, double tol, void* stream, Prof& P);
int launch_assemble_interface(const Tables& t, const DeviceTables& d, const Layout& L, char* ws,
                              void* stream, Prof& P);
int launch_solve_interface(const Tables& t, const DeviceTables& d, const Layout& L, char* ws,
                           double* X, void* stream, Prof& P);
int configure_local(const Tables& t, DeviceTables& d);
int configure_interface(const Tables& t, DeviceTables& d);
int configure_reconstruct(const Tables& t);
int autotune_local(const Tables& t, DeviceTables& d, const Layout& L, char* ws, const double* f,
                   void* stream, int reps, int* best_solve, int* best_sweep, int* best_factor, int* best_factor_mid,
                   float* ms_out);
int launch_postprocess(const Tables& t, const DeviceTables& d, const Layout& L, char* ws, const double* u,
                       double* u_out, double* mres, const double* f, int precision, int sweeps, double tol,
                       void* stream, Prof& P);
int launch_local_finish(const Tables& t, const DeviceTables& d, const Layout& L, char* ws, const double* f,
                        void* stream, Prof& P);
int launch_reconstruct(const Tables& t, const DeviceTables& d, const Layout& L, char* ws,
                       const double* X, double* p, double* u, double* mres, const double* K,
                       const double* f, void* stream, Prof& P);
}
