// Internal declarations of the IgA-SGBEM GB300 library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/igs.h"

namespace igs {

constexpr int kMaxDegree = 5;
constexpr int kMaxNref = 4;
constexpr int kMaxGeomDegree = 7;
constexpr int kGaussRhs = 8;          // Gauss points per refined element for the b2 inner rule
constexpr int kTreeMaxLevels = 30;    // levels of the double-layer treecode (MIXED tier)
constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
std::string cuda_msg(cudaError_t e, const char* what, const char* file, int line);

#define IGS_CUDA(call)                                                           \
    do {                                                                          \
        cudaError_t _e = (call);                                                  \
        if (_e != cudaSuccess) {                                                  \
            throw ::igs::Error(IGS_E_CUDA, ::igs::cuda_msg(_e, #call, __FILE__, __LINE__)); \
        }                                                                         \
    } while (0)

struct Error {
    int code;
    std::string msg;
    Error(int c, std::string m) : code(c), msg(std::move(m)) {}
};

// ------------------------------------------------------------------ plan
// Integer description of the discretisation (Sect. 3-4).  Node positions are
// kept in units of h_f / den with den = 2 (d + 1), so every node of Sect. 4
// (d+2 uniform points in the first and last refined element, midpoints and
// breakpoints elsewhere) has an integer position.
struct Plan {
    int n = 0, d = 0, Nh = 0, Nref = 0, M = 0, Nq = 0, NE = 0, closed = 0;
    int den = 0;
    double a = 0, b = 0, L = 0, h = 0, hf = 0;
    std::vector<int> pos_num;     // [Nq]   position * den (units of h_f)
    std::vector<int> jfirst;      // [Nq]   first test function (unrolled) whose band holds the node
    std::vector<int> member;      // [Nq]   bit r set if B_{jfirst+r}(eta) != 0
    std::vector<int> fspan;       // [Nq]   refined element holding the node (0..M-1)
    std::vector<int> lo, hi;      // [n]    unrolled node range of N^(i)
    std::vector<int> jlo1, jhi1, jlo2, jhi2;  // [n] exactness functions J^(i) (1-2 ranges)
    std::vector<int> elo1, ehi1, elo2, ehi2;  // [n] refined elements of supp(B_i) (half-open)
    std::vector<int> gfirst, glast;           // [NE] node range touching supp(B-bar_j)
    int max_nodes_i = 0, max_fine_i = 0;      // largest |N^(i)|, |J^(i)|
    int max_tile_nodes = 0;                   // largest node range of a row tile
    std::vector<double> piece;    // [(d+1)*(d+1)] cardinal B-spline pieces: N_d(l+u) = sum_k piece[l*(d+1)+k] u^k
    std::vector<double> series;   // [(d+1)*kSeries] far-field log series coefficients
};
constexpr int kSeries = 30;

int build_plan(Plan& p, double a, double b, int Nh, int d, int Nref, int closed, std::string& err);
int collocation_nodes(const Plan& P, std::vector<int>& out, std::string& err);

}  // namespace igs

// ------------------------------------------------------------------ handles
struct igs_ctx_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int live_geoms = 0, live_probs = 0, live_batches = 0;
};

struct igs_geom_s {
    igs_ctx ctx = nullptr;
    int degree = 0, n_ctrl = 0, n_knots = 0, closed = 0, rational = 0;
    double a = 0, b = 0;
    double* d_knots = nullptr;
    double* d_ctrl = nullptr;    // n_ctrl x 2
    double* d_w = nullptr;       // n_ctrl (all ones for a B-spline)
    int live_probs = 0;
};

struct igs_prob_s {
    igs_geom geom = nullptr;
    igs::Plan plan;
    int precision = IGS_FP64;
    int rules_ready = 0, geometry_ready = 0, assembled = 0, factored = 0;
    int live_batches = 0;         // batches that reference this problem
    int64_t bytes = 0;
    igs_timing timing{};
    int launches = 0;

    // plan arrays on device
    int *d_pos = nullptr, *d_jfirst = nullptr, *d_member = nullptr, *d_fspan = nullptr;
    int *d_lo = nullptr, *d_hi = nullptr;
    int *d_jr = nullptr;          // [n][8]: jlo1,jhi1,jlo2,jhi2,elo1,ehi1,elo2,ehi2
    int *d_gfirst = nullptr, *d_glast = nullptr;
    double *d_piece = nullptr, *d_series = nullptr;

    // rules (FP64)
    double* d_eta = nullptr;      // [Nq]
    double* d_Bf = nullptr;       // [Nq][d+1] exactness functions e..e+d at the node (e = fspan)
    double* d_Bt = nullptr;       // [Nq][d+1] test functions jfirst..jfirst+d at the node
    double* d_W = nullptr;        // [Nq][d+1] regular weights w^(jfirst+r)_m
    double* d_G = nullptr;        // [NE][d+1] Cholesky factor of G (row j: L(j, j-r))
    double* d_Z = nullptr;        // [NE][Nq] G^{-1} mu(eta_m) (work)
    // Singular rules W^s[m][m'] (row m = w^{eta_m}).  Column m' is stored
    // explicitly for the ws_B columns at each end (ws_B = n_quad: dense); the
    // interior is 2-periodic Toeplitz (ws_T[p][m - m' + n_quad - 1], p =
    // (m' - ws_B) & 1) except for the ws_R rows at each end (ws_row).
    int ws_B = 0, ws_R = 0;
    double* d_WsT = nullptr;      // [2 ws_B][Nq] boundary columns: d_WsT[c][m] = W^s[m][m'(c)]
    float* d_WsT32 = nullptr;     // FP32 copy (MIXED tier)
    double* d_WsRow = nullptr;    // [2 ws_R][Nq] boundary rows: d_WsRow[r][m'] = W^s[m(r)][m']
    float* d_WsRow32 = nullptr;
    double* d_WsToe = nullptr;    // [2][2 Nq - 1] interior Toeplitz sequences
    float* d_WsToe32 = nullptr;
    int* d_flag = nullptr;        // device status word

    // geometry at nodes
    double* d_geo = nullptr;      // [5][Nq]: x, y, x', y', J
    void* d_nodes = nullptr;      // tier-specific node records
    void* d_P = nullptr;          // [Nq][d+1] J * W (tier type)
    void* d_Q = nullptr;          // [Nq][d+1] J * B_test (tier type)

    // matrix and solve
    void* d_A = nullptr;          // [n][n] tier type (row-major)
    void* d_AT = nullptr;         // [n][n] A^T in the tier type, written by the assembly for the symmetrisation
    int at_ready = 0;             // d_AT holds the transpose of the current A
    void* d_F = nullptr;          // [n][n] Cholesky factor (tier type): lower = L, upper = L^T
    void* d_diagL = nullptr;      // [n][64] factored diagonal blocks of L (tier type)
    void* d_diagLinv = nullptr;   // [n][64] inverses of the diagonal blocks of L (tier type)
    float* d_diagLinv128 = nullptr;  // [n][128] inverses of the 128-row diagonal blocks (MIXED tier)
    cudaGraphExec_t factor_exec = nullptr;   // captured factorisation (fixed pointers and sizes)
    cudaEvent_t asm_ev[3] = {nullptr, nullptr, nullptr};   // geometry / assembly events of the last igs_assemble
    bool asm_pending = false;     // those events not yet read into timing
    int factor_runs = 0;                     // factorisations so far (the graph is captured from the second)
    int* d_tflags = nullptr;      // [n/64] per-block completion flags of the triangular solves
    unsigned long long* d_tpub = nullptr;  // [8][n] published FP32 solution words (value, epoch)
    float* d_timg = nullptr;      // two outer blocks of split factor columns (MIXED tier, n >= 4096)
    int tepoch = 0;               // flag value of the current triangular solve
    cudaStream_t aux_stream = nullptr;   // right-hand side beside the factorisation (igs_solve_data)
    bool coop_ok = false;         // cooperative launch available
    double* d_As64 = nullptr;     // (A+A^T)/2 in FP64 for the refinement residuals (FP64 tier)
    float* d_dscale = nullptr;    // [n] As_ii^-1/2: the MIXED factor is that of D As D
    int rhs_n = 0;
    double* d_beta = nullptr;     // [nrhs][n]
    double* d_rhs_geo = nullptr;  // [5][Ng] geometry at the rhs Gauss points
    double* d_rhs_w = nullptr;    // [Ng] Gauss weights
    double* d_rhs_t = nullptr;    // [Ng] Gauss abscissae
    int Ng = 0;
    // treecode of the double-layer sum (MIXED tier, closed curves): clusters of
    // the rhs Gauss points, level 0 = leaves; geometry in one buffer
    int tree_L = 0, tree_C = 0;
    int tree_off[igs::kTreeMaxLevels] = {}, tree_cnt[igs::kTreeMaxLevels] = {};
    void* d_tree = nullptr;
};

namespace igs {
// Read access to the singular rules in either layout (see igs_prob_s).
template <typename T>
struct WsView {
    const T* col;
    const T* row;
    const T* toe;
    int Nq, B, R;
};
// W^s[ma][mb]: weight of node mb in the singular rule at node ma.
template <typename T>
__host__ __device__ __forceinline__ T ws_at(const WsView<T>& v, int ma, int mb) {
    if (mb < v.B) return v.col[(size_t)mb * v.Nq + ma];
    if (mb >= v.Nq - v.B) return v.col[(size_t)(mb - v.Nq + 2 * v.B) * v.Nq + ma];
    if (ma < v.R) return v.row[(size_t)ma * v.Nq + mb];
    if (ma >= v.Nq - v.R) return v.row[(size_t)(ma - v.Nq + 2 * v.R) * v.Nq + mb];
    return v.toe[(size_t)((mb - v.B) & 1) * (2 * (size_t)v.Nq - 1) + (ma - mb + v.Nq - 1)];
}

#ifdef __CUDACC__
// The PTX approximate base-2 logarithm and quotient with subnormal inputs and
// results flushed to zero: one special-function instruction (and one multiply
// for the quotient), without the rescaling a subnormal-preserving form adds.
// Every argument these kernels pass is a normal number (squared distances and
// parameter differences of distinct nodes), where both agree with the
// subnormal-preserving forms bit for bit.
__device__ __forceinline__ float lg2_ftz(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float div_ftz(float x, float y) {
    float r;
    asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(x), "f"(y));
    return r;
}
#endif
}  // namespace igs

namespace igs {
// allocation helpers (stream-ordered, accounted on the problem)
void* dev_alloc(igs_prob p, size_t bytes);
void dev_free_raw(igs_prob p, void* ptr);
template <typename T>
inline void dev_free(igs_prob p, T*& ptr) {
    if (ptr) dev_free_raw(p, (void*)ptr);
    ptr = nullptr;
}

// phases (implemented in the .cu files)
void rules_build(igs_prob p);
void ws_expand(igs_prob p, double* d_out);   // dense W^s[m][m'] into d_out[Nq][Nq]
void geometry_eval(igs_geom g, const double* d_t, int count, double* d_out, cudaStream_t s);
void geometry_nodes(igs_prob p);
void assemble_matrix(igs_prob p);
void rhs_prepare(igs_prob p);
void rhs_tree_geometry(igs_prob p, cudaStream_t s);   // treecode clusters after a geometry change
void rhs_build(igs_prob p, const double* d_uD, int nrhs);
void rhs_build_noalloc(igs_prob p, const double* d_uD, int nrhs, double* d_beta);
int rhs_slots(const igs_prob p);   // scratch slots (each nrhs x N_quad doubles) of the node potentials
void rhs_node_potentials(igs_prob p, const double* d_uD, int nrhs, double* scratch, const double** vsum, int* np,
                         cudaStream_t s);
void rhs_compute(igs_prob p, const double* d_uD, int nrhs, double* d_beta, double* scratch, cudaStream_t s);
void solve_with_data(igs_prob p, const double* d_uD, int nrhs, double* d_alpha, double* resid);
void collocation_solve(igs_prob p, const double* d_uD, int nrhs, double* d_alpha, double* Ac_out, int ac_mem,
                       int* nodes_out);
void potential_eval(igs_prob p, const double* d_alpha, const double* d_uD, int nrhs, const double* d_xy,
                    int64_t count, double* d_u);
void solve_system(igs_prob p, double* d_beta, int nrhs, double* d_alpha, double* resid);
double measure_peak(int device, int kind, double* ms);    // rate of one pipe (peaks.cu)
int wait_selftest(int device, double budget_s);   // 1: the bounded wait gave up
}  // namespace igs

// ------------------------------------------------------------- FP32 assembly
namespace igs {
// Coordinates x, y and parameter offsets e = eta - eta_0, eb = L - e, each
// divided by L and held as float-float (hi, lo) pairs; ln J.
struct NodeF { float xh, xl, yh, yl, eh, el, ebh, ebl, lnJ; };

// One problem's FP32 assembly inputs (device pointers).
struct TileF {
    int n, Nq;
    const int* lo;
    const int* hi;
    const int* jfirst;
    const NodeF* nodes;
    const float* P;
    const float* Q;
    WsView<float> ws;
    float* A;
    float* AT;           // A^T (row-major, same ld), written beside A when not NULL
    int64_t ld;
    int maxr;
};

// Batched form: per-problem tile inputs and geometry/prep inputs.
struct BatchItemF {
    TileF t;
    int d, closed, nt;
};
struct BatchGeomF {
    int gdeg, nb;
    const double* knots;
    const double* ctrl;
    const double* w;
    const double* eta;
    int Nq, d;
    double L;
    const double* W;
    const double* Bt;
    double* geo;
    NodeF* nodes;
    float* P;
    float* Q;
    int node0;
};

int max_tile_range(const Plan& P, int TI);
size_t tile_smem_f(int maxr, int d, int TI);
TileF tile_args_f(igs_prob p, int maxr);
void batch_geom_f(const BatchGeomF* d_items, int nitems, int total, cudaStream_t s);
int batch_blocks_per_sm(int TI, int threads, size_t smem);
void batch_assemble_f(int TI, const BatchItemF* d_items, const int2* d_units, int nunits, int* d_counter, int grid,
                      int threads, size_t smem, cudaStream_t s);
}  // namespace igs

// ------------------------------------------------------- C-ABI entry helpers
namespace igs {
// Raise a kernel's dynamic shared-memory limit to at least `bytes`; the limit
// only grows, under a lock, so that concurrent callers needing different
// amounts never lower it between another caller's setting and its launch.
void ensure_dyn_smem(const void* func, size_t bytes);
void set_error(const std::string& msg);
void ensure_rules(igs_prob p);
void ensure_geometry(igs_prob p);
}  // namespace igs

#define API_BEGIN \
    try {
#define API_END                                                               \
    }                                                                         \
    catch (const igs::Error& e) {                                             \
        igs::set_error(e.msg);                                                \
        return e.code;                                                        \
    }                                                                         \
    catch (const std::bad_alloc&) {                                           \
        igs::set_error("host allocation failed");                             \
        return IGS_E_NO_MEMORY;                                               \
    }                                                                         \
    catch (...) {                                                             \
        igs::set_error("unexpected error");                                   \
        return IGS_E_CUDA;                                                    \
    }                                                                         \
    return IGS_OK;

#define REQUIRE(cond, code, msg)                      \
    do {                                              \
        if (!(cond)) throw igs::Error((code), (msg)); \
    } while (0)
