// pmg_internal.h -- internal data structures of libpmgfr.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/pmgfr.h"
#include "physics_dw.cuh"
#include "tma.cuh"

namespace pmg {

constexpr int kMaxP = 5;
constexpr int kMaxLevels = 8;

// Storage type W of the factored block inverses and the arithmetic type of
// their application, Blk<W>::acc: FP64 and FP32 blocks are applied in their
// own precision, BF16 blocks (8-bit significand, FP32 exponent range) with
// FP32 accumulation.
template <class W> struct Blk { using acc = W; };
template <> struct Blk<__nv_bfloat16> { using acc = float; };

// Block scales are powers of two, so applying them in the block arithmetic
// after the conversion gives the same value (barring under- or overflow) and,
// for FP32 and BF16 blocks, keeps these multiplications off the FP64 pipe.
template <class W>
__device__ __forceinline__ typename Blk<W>::acc scaled_in(double x, double s) {
  using A = typename Blk<W>::acc;
  return (A)x * (A)s;
}
template <class W>
__device__ __forceinline__ double scaled_out(typename Blk<W>::acc a, double s) {
  using A = typename Blk<W>::acc;
  return (double)(a * (A)s);
}
// One stored block entry in the arithmetic type.
__device__ __forceinline__ double blk_val(double x) { return x; }
__device__ __forceinline__ float blk_val(float x) { return x; }
__device__ __forceinline__ float blk_val(__nv_bfloat16 x) { return __bfloat162float(x); }

// ----------------------------------------------------------------- host side
struct Ref1D {
  int P;
  std::vector<double> x, w, D, lm, lp, gL, gR;
};

struct FaceRec {
  int eL, fL, eR, fR, rev;
};

struct MeshHost {
  int E = 0, Ng = 0;
  std::vector<double> nodes;
  std::vector<int> nbr;
  std::vector<FaceRec> faces;
};

// Tiles of the multi-sweep smoother (host_tables.cpp build_tiles).
struct TileSet {
  int depth = 0, n_tiles = 0, max_elems = 0;
  std::vector<int> off;        // n_tiles + 1 offsets into elems
  std::vector<int> layer_end;  // n_tiles x (depth + 1): end of the core, then of halo layers 1..depth
  std::vector<int> elems;      // element ids, per tile core first, then halo layers
  std::vector<int> lnbr;       // per listed element and face: slot of the neighbour in the tile (-1: outside)
};
TileSet build_tiles(const struct MeshHost& m, int core, int depth);

struct LevelGeomHost {
  std::vector<double> met;   // 5 planes of E*N: a, b, c, d, 1/|J|
  std::vector<double> xy;    // (E, N, 2)
  std::vector<double> face;  // (E, 4, n1, 3): unit outward normal, area factor
  std::vector<double> fJinv; // (E, 4, n1) or (E, 6, NF): 1/|J| at the face points
};

Ref1D make_ref1d(int P);
void make_transfer(const Ref1D& f, const Ref1D& c, std::vector<double>& R, std::vector<double>& I);
void build_faces(MeshHost& m);
void build_level_geometry(const MeshHost& m, const Ref1D& r, LevelGeomHost& g);
// Hexahedra (host_tables3.cpp): face list with orientation codes in FaceRec.rev,
// metric planes (J a^i_n, then 1/J), coordinates (E, N, 3), face geometry
// (E, 6, NF, 4: unit outward normal, area).
void build_faces3(MeshHost& m);
void build_level_geometry3(const MeshHost& m, const Ref1D& r, LevelGeomHost& g);
std::vector<double> element_sizes(const MeshHost& m);

// --------------------------------------------------------------- device side
// Operator tables of one level, passed to kernels by value.
struct OpTab {
  double D[kMaxP + 1][kMaxP + 1];
  double lm[kMaxP + 1], lp[kMaxP + 1], gL[kMaxP + 1], gR[kMaxP + 1];
  double pen;   // BR2 lifting factor eta_f g_R'(1) = 4 (P+1)^2 / 2
};

// Restriction (nc x nf) and prolongation (nf x nc) 1D operators, by value.
struct XferTab {
  double R[kMaxP + 1][kMaxP + 1];
  double I[kMaxP + 1][kMaxP + 1];
};

struct LevelDev {
  int level = 0;               // index in the hierarchy (0: finest)
  int P = 0, n1 = 0, N = 0, n = 0;
  int NF = 0;                  // points per face: P + 1 (2D), (P + 1)^2 (3D)
  size_t tot = 0;              // nv * E * N
  OpTab op;
  OpTabW opw;                  // the same operators in double-word
  double* q = nullptr;         // state
  double* q2 = nullptr;        // second state buffer of fused (ping-pong) sweeps
  bool fused = false;          // coarse level smoothed by the fused one-launch sweep
  double* qb = nullptr;        // state at entry of the level in the V-cycle
  double* S = nullptr;         // FAS forcing
  double* F = nullptr;         // level system residual F_l(q) - S_l
  double* Cgauge = nullptr;    // gauge storage on a level with P < geometry order: p_gauge times the
                               // level's discrete metric-identity residual (momentum rows), the part of
                               // R that the gauge momentum flux leaves out; a constant, so the FAS
                               // coarse-level equations F_c(q) - F_c(q^b) - P d do not see it, and the
                               // residual calls add it back
  double* Pd = nullptr;        // restricted defect (coarse levels)
  double* met = nullptr;       // 5 * E * N (2D), 10 * E * N (3D)
  double* face = nullptr;      // E * 4 * n1 * 3 (2D), E * 6 * NF * 4 (3D)
  double* Fcom = nullptr;      // nv * E * faces * NF common fluxes, outward
  // viscous terms (mu > 0 only); hexahedra in brackets
  double* Gb = nullptr;        // 6 [12] * E * N broken gradients of (u, v, T) [(u, v, w, T)]:
                               // x planes, then y [, then z]
  double* Qj = nullptr;        // 3 * E * 4 * n1 [4 * E * 6 * NF]: q_com - q_own of the same
                               // variables at each element face point
  double* fJinv = nullptr;     // E * 4 * n1 [E * 6 * NF]: 1/|J| at the face points
  double* Dfull = nullptr;     // E * n * n assembled FP64 blocks (row-major)
  void* Dinv = nullptr;        // E * n * n factored inverse (column-major), FP32 or FP64
  double* rs = nullptr;        // E * n row scales
  double* cs = nullptr;        // E * n column scales
  bool assembled = false, factored = false;
  // multi-sweep tiles (k_tile.cu), when the level is tiled
  bool tileable = false;       // the double-word fused sweep and tiles may serve this level
  bool tiled = false;
  int n_tiles = 0, tile_M = 0, tile_depth = 0, tile_core = 0;
  int* d_toff = nullptr;       // n_tiles + 1
  int* d_tlayer = nullptr;     // n_tiles * (tile_depth + 1)
  int* d_telems = nullptr;     // listed elements of all tiles
  int* d_tlnbr = nullptr;      // 4 per listed element
};

// Residual kernel epilogues.
enum ResMode : int {
  RES_PURE = 0,     // out = R
  RES_SYSTEM = 1,   // out = -q_c/(omega dt) + R (+ src) - S   (level system residual)
  RES_FORCING = 2,  // S = -q_c/(omega dt) + R + Pd;  out = -Pd
  RES_STAGEF = 3    // out = -q_c/(omega dt) + R (+ src), no S
};

// Kernel classes timed by the optional per-launch event profiler.
enum KClass : int { K_FACE = 0, K_VOLUME, K_APPLY, K_ASSEMBLE, K_FACTOR, K_RESTRICT, K_PROLONG, K_NORM, K_STAGE,
                    K_FUSED, K_COUNT };

// Device-side stage loop (k_loop.cu): its state in device memory and its
// fixed parameters.
enum LoopStatus : int { LOOP_RUNNING = 0, LOOP_CONVERGED, LOOP_NONFINITE, LOOP_NOTCONV, LOOP_SINGULAR, LOOP_TIMEOUT };
struct LoopState {
  double n0, prev, dtau, built, dtau_max, final_norm;
  int m, iters, status, n_refresh;
};
struct LoopParams {
  double tol;
  int refresh_every, refresh_always, max_pseudo;
};

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;       // pairs (start, end)
  std::vector<int> tag;              // class * kMaxLevels + level of each pair
  int used = 0;                      // pairs recorded since the last harvest
  double ms[K_COUNT][kMaxLevels] = {};
  long long count[K_COUNT][kMaxLevels] = {};
};

struct Ctx {
  pmg_config cfg;
  int dim = 2, nv = 4, nfc = 4;   // dimension, working variables, faces per element
  Profiler prof;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  Phys ph;
  PhysW phw;                   // double-word copies of the gas constants
  MeshHost mesh;
  bool mesh_ready = false;
  int E = 0, n_faces = 0;
  int* d_faces = nullptr;      // n_faces * 5
  double* d_dx = nullptr;      // E element sizes of the CFL form
  LevelDev lev[kMaxLevels];
  std::vector<double> xy_host[kMaxLevels];   // solution point coordinates of each level
  XferTab xfer[kMaxLevels];
  // stage data (finest level)
  double* src = nullptr;
  double* qn = nullptr;        // state at the start of the physical step
  double* qcn = nullptr;       // conservative state at the start of the step
  double* Rst[6] = {nullptr};  // R(q^j) of the stages
  double omega_dt = 1.0;
  bool stage_ready = false;
  bool split_stage = false;    // src holds sum_j a_ij R^j / omega and q^n is in qn
  std::vector<double> hist_norm, hist_dtau;   // pseudo-iteration history of the last step
  bool F0_valid = false;       // lev[0].F holds F_0(q) for the current q
  // Newton-Krylov stage solver (api.cu nk_stage_solve; vectors of the finest size)
  int stage_solver = PMG_STAGE_PTC;
  pmg_nk_options nk{};
  int nk_m = 0;                // Krylov vectors allocated for
  double* nk_q = nullptr;      // Newton iterate
  double* nk_F = nullptr;      // F at the iterate
  double* nk_src = nullptr;    // the stage source (the V-cycle preconditioner changes c.src)
  double* nk_w = nullptr;      // A z, and the restart residual
  double* nk_t = nullptr;      // scratch
  double* nk_x = nullptr;      // Newton correction
  double* nk_V = nullptr;      // (m + 1) Krylov basis vectors
  double* nk_Z = nullptr;      // m preconditioned directions
  double* nk_part = nullptr;   // partial sums of the multi-dot kernel
  double* nk_dots = nullptr;   // its results (3 m + 3)
  double* nk_coef = nullptr;   // combination coefficients (m)
  double* h_nk = nullptr;      // pinned host mirror (3 m + 3)
  long long nk_count[4] = {0, 0, 0, 0};   // newton, krylov, vcycles, residuals
  // reductions
  double* d_partial = nullptr; // per-block partial sums
  int n_partial = 0;
  double* d_scal = nullptr;    // device scalars: [0] ||F||^2, [1] status flags
  double* h_scal = nullptr;    // pinned host mirror
  int* d_flag = nullptr;       // singular-pivot / error flags
  // scratch vectors for API calls with host or device I/O
  double* d_tmp0 = nullptr;
  double* d_tmp1 = nullptr;
  size_t tmp_size = 0;
  // CUDA graphs of the V-cycle (0: plain, 1: with refresh), built for one
  // omega dt and one stage form (split_stage)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  double graph_inv_odt[2] = {0.0, 0.0};
  int graph_split[2] = {-1, -1};
  // device-side stage loop (cfg.device_loop): the WHILE graph, its state
  cudaGraphExec_t loop_exec = nullptr;
  double loop_inv_odt = 0.0;
  int loop_split = -1;
  LoopState* d_loop = nullptr;
  LoopState* h_loop = nullptr;      // pinned mirror
  double* d_hist = nullptr;         // 2 (max_pseudo + 1): norms, then dtau
  double* h_hist = nullptr;         // pinned mirror
  double* d_dtau = nullptr;    // pseudo time step read by the assembly kernel
  double* h_dtau = nullptr;
  // ESDIRK3 tableau
  double A[6][6], b[6], c[6];
  int stages = 4;
};

// Residual arithmetic (pmg_config.flux_prec): double-word in a residual
// evaluation of a coarse level (and of the finest for PMG_FLUX_DW) ...
inline bool flux_dw(const Ctx& c, const LevelDev& L) {
  return c.cfg.flux_prec == PMG_FLUX_DW || (c.cfg.flux_prec == PMG_FLUX_DW_SMOOTH && L.level > 0);
}
// ... and in every element-Jacobi sweep unless PMG_FLUX_FP64.
inline bool flux_dw_sweep(const Ctx& c) { return c.cfg.flux_prec != PMG_FLUX_FP64; }

// ---------------------------------------------------------- kernel launchers
// sweep: the flux of an element-Jacobi sweep (flux_dw_sweep) rather than of
// a residual evaluation (flux_dw)
void launch_face_flux(const Ctx& c, const LevelDev& L, const double* q, cudaStream_t s, bool sweep = false);
cudaError_t prepare_residual_kernels(const Ctx& c);   // once per mesh upload
// Residual-and-update sweep in double-word arithmetic (k_volume_dw.cu):
// used where volume_dw_applies().
bool volume_dw_applies(const Ctx& c);
void launch_volume_apply_dw(const Ctx& c, const LevelDev& L, double* q, double inv_odt, const double* src,
                            const double* S, const double* qref, int prec, cudaStream_t s);
cudaError_t prepare_volume_dw_kernels(const Ctx& c);
void launch_volume(const Ctx& c, const LevelDev& L, int level, const double* q, double* out, ResMode mode,
                   double inv_odt, const double* src, const double* S, double* Sout, const double* Pd,
                   double* partial, cudaStream_t s, const double* qn = nullptr);
void launch_norm_final(const double* partial, int n, double* out, cudaStream_t s);
void launch_volume_apply(const Ctx& c, const LevelDev& L, double* q, double inv_odt, const double* src,
                         const double* S, const double* qn, int prec, cudaStream_t s);
void launch_assemble(const Ctx& c, const LevelDev& L, const double* q, const double* d_dtau, double inv_odt,
                     cudaStream_t s);
void launch_factor(const Ctx& c, LevelDev& L, int level, int prec, int* flag, cudaStream_t s);
void launch_apply(const Ctx& c, const LevelDev& L, int prec, const double* r, double* x, int accumulate,
                  cudaStream_t s);
void launch_restrict(const Ctx& c, const LevelDev& Lf, const LevelDev& Lc, const XferTab& X, const double* in,
                     double* out, double* out2, double scale, cudaStream_t s);
void launch_prolong_add(const Ctx& c, const LevelDev& Lf, const LevelDev& Lc, const XferTab& X, const double* qc,
                        const double* qcb, double* qf, cudaStream_t s);
void launch_prolong(const Ctx& c, const LevelDev& Lf, const LevelDev& Lc, const XferTab& X, const double* in,
                    double* out, cudaStream_t s);
void launch_cons(const Ctx& c, int N, const double* q, double* qc, cudaStream_t s);
void launch_stage_src(const Ctx& c, int N, const double* qcn, double* const* R, const double* a, int nr,
                      double dt, double inv_odt, double* src, cudaStream_t s);
void launch_bsum_update(const Ctx& c, int N, const double* qn, double* const* R, const double* b, int nr,
                        double dt, double* q, cudaStream_t s);
void launch_shift_pressure(size_t plane, double delta, double* q, cudaStream_t s);
void launch_dtau_min(const Ctx& c, double* partial, double* out, cudaStream_t s);
void launch_grad(const Ctx& c, const LevelDev& L, const double* q, cudaStream_t s);
void launch_assemble_visc(const Ctx& c, const LevelDev& L, const double* q, cudaStream_t s);
void launch_fused_sweep(const Ctx& c, const LevelDev& L, const double* qin, double* qout, double inv_odt,
                        const double* src, const double* S, const double* qref, int prec, cudaStream_t s);
void launch_loop_controller(LoopState* st, const double* scal, int* sing_flag, double* d_dtau, double* hist_norm,
                            double* hist_dtau, const LoopParams& prm, cudaGraphConditionalHandle h_loop,
                            cudaGraphConditionalHandle h_refresh, cudaGraphConditionalHandle h_plain,
                            cudaStream_t s);
// Hexahedral kernels (k3_*.cu); the launchers above dispatch to them when dim = 3.
void launch_face_flux3(const Ctx& c, const LevelDev& L, const double* q, cudaStream_t s);
void launch_volume3(const Ctx& c, const LevelDev& L, const double* q, double* out, ResMode mode, double inv_odt,
                    const double* src, const double* S, double* Sout, const double* Pd, double* partial,
                    cudaStream_t s, const double* qn);
void launch_volume_apply3(const Ctx& c, const LevelDev& L, double* q, double inv_odt, const double* src,
                          const double* S, const double* qn, int prec, cudaStream_t s);
int residual_blocks_for3(int P, int E);
void launch_assemble3(const Ctx& c, const LevelDev& L, const double* q, const double* d_dtau, double inv_odt,
                      cudaStream_t s);
// viscous terms on hexahedra: broken gradients (Gb, 12 planes) and the
// viscous part of the element blocks (k3_viscous.cu)
void launch_grad3(const Ctx& c, const LevelDev& L, const double* q, cudaStream_t s);
void launch_assemble_visc3(const Ctx& c, const LevelDev& L, const double* q, cudaStream_t s);
cudaError_t prepare_assemble_visc3();
void launch_apply3(const Ctx& c, const LevelDev& L, int prec, const double* r, double* x, int accumulate,
                   cudaStream_t s);
cudaError_t prepare_kernels3(const Ctx& c);
void launch_restrict3(const Ctx& c, const LevelDev& Lf, const LevelDev& Lc, const XferTab& X, const double* in,
                      double* out, double* out2, double scale, cudaStream_t s);
void launch_prolong3(const Ctx& c, const LevelDev& Lf, const LevelDev& Lc, const XferTab& X, const double* qc,
                     const double* qcb, double* qf, int add, cudaStream_t s);
void launch_bsum_update3(const Ctx& c, int N, const double* qn, double* const* R, const double* b, int nr,
                         double dt, double* q, cudaStream_t s);
// Vector kernels of the Newton-Krylov solver (k_krylov.cu).
constexpr int kDotBlocks = 304;
struct Scale5 {
  double s[5];
};
// out_j = sum_i X_j[i] y[i] for j < k, X_j = X + j ld (part: kDotBlocks k doubles)
void launch_multi_dot(const double* X, size_t ld, int k, const double* y, size_t n, double* part, double* out,
                      cudaStream_t s);
// y += sign sum_{j<k} coef[j] X_j (coef on the device, k <= 64)
void launch_combination(double* y, const double* X, size_t ld, int k, const double* coef, double sign, size_t n,
                        cudaStream_t s);
// out = (a0 x0 + a1 x1) s0[v] + a2 x2 s2[v], v = i / plane (null inputs count as 0)
void launch_plane_combine(double* out, const double* x0, double a0, const double* x1, double a1, const Scale5& s0,
                          const double* x2, double a2, const Scale5& s2, size_t plane, size_t n, cudaStream_t s);
// out += a w_v (Gamma(q) z)_v at every point (q stored with p - p_ref)
void launch_gamma_apply(int nv, size_t plane, const double* q, const double* z, double* out, double a,
                        const Scale5& w, const Phys& ph, cudaStream_t s);
// max over the p and T planes of |dx| / |x (+ p_ref for p)| into out[0]
void launch_rel_change(const double* x, const double* dx, size_t plane, int tslot, double p_ref, double* part,
                       double* out, cudaStream_t s);
void launch_tile_sweeps(const Ctx& c, const LevelDev& L, const double* qin, double* qout, int nsweep,
                        double inv_odt, const double* S, const double* qref, int prec, cudaStream_t s);
size_t tile_smem_bytes(int P, int prec, int M);
int tile_face_points(int P);
cudaError_t prepare_tile_kernel(int P, int prec, size_t bytes);
int residual_threads_per_block(int P);
int residual_blocks_for(int P, int E);
cudaError_t prepare_kernels(const Ctx& c);
int factor_max_n(int prec);
// Blocks larger than one CTA's shared memory (k_factor_cluster.cu): CTAs per
// block (1: the one-CTA kernel; 2, 4, 8: a cluster; 0: too large).
int factor_cluster_size(int n, int prec);
size_t factor_cluster_smem(int n, int C, int tbytes);
void launch_factor_cluster(const Ctx& c, LevelDev& L, int level, int prec, int C, int* flag, cudaStream_t s);
cudaError_t prepare_factor_cluster(int n, int prec, int C);

}  // namespace pmg
