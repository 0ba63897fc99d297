// Internal declarations of libmclbm (GB300 / sm_103a). Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "mclbm.h"

namespace mcl {

constexpr int kQ = 9;        // D2Q9 directions (Eq 21)
constexpr int kPlanes = 27;  // f^w, f^p, g (one thermal set)
constexpr int kPlanes2 = 36; // f^w, f^p, g^w, g^p (two thermal sets)
constexpr int kFields = 10;  // MCLBM_UX ... MCLBM_THETA_P
constexpr uint32_t kFieldMask = (1u << kFields) - 1u;
constexpr int kGraphSteps = 64;     // steps per captured batch graph (even: the buffers come back)
constexpr int kGraphLogMax = 10;    // single cavity: graphs of 2^k steps, k = 1 .. kGraphLogMax
constexpr int kMaxRedBlocks = 304;  // reduction partials: 2 CTAs per SM on 152 SMs
constexpr int kRedWidth = 8;        // doubles per reduction partial

// FP32 constants of one step, folded on the host from the FP64 create-time constants.
// Force coefficients turn lattice moments directly into lattice force densities.
struct StepConsts {
  float rho_w0, rho_p0;       // initial partial densities: offsets of the stored deviations
  float inv_tau_w, inv_tau_p; // 1 / momentum relaxation times (Eqs 22-23)
  float tau_tw, tau_tp;       // thermal relaxation times of the components (Eq 24)
  float buoy;                 // (beta_ns / beta_f) G_B: buoyancy per unit rho theta (Eq 2, Eq 20)
  float gG;                   // (1 - rho_f / rho_p) g_lb: gravity minus buoyancy per unit rho^p
  float phi_per_rho_p;        // rho_f / rho_p: volume fraction per unit particle partial density
  float cB;                   // Brownian: F_B = -cB rho^p (T/T0)^2 grad rho^p
  float cT;                   // thermophoresis: F_T = -cT rho^p grad theta / (T/T0)
  float cS;                   // Saffman: F_S = cS rho^p |u^p|^(1/2) R90(u^w - u^p)
  float cM;                   // Magnus: F_M = cM rho^p |u^w + u^p|^2 zeta(z) n_wall
  float t_ratio;              // dT / T0: T/T0 = 1 + theta dT / T0
  float beta_dt;              // beta_St dt: Stokes drag rate per step
  float cRe;                  // Re_d = cRe |u^w - u^p|
  float two_over_ny;          // 2 z / H = two_over_ny * z_lattice
  float inv_nx;               // 1 / nx: slope of the conduction profile theta_c
  float th_c0;                // theta_c(0) = 1/2 - 1/(2 nx); theta_c(i) = th_c0 - i / nx
  uint32_t mask;              // MCLBM_F_* bits
  int has_p;                  // initial phi > 0
  int two_sets;               // two thermal population sets (g^w, g^p)
  float r_cp;                 // C_p,p / C_p,f: the heat-capacity weight of Eq 33
  double rho_w0_d, rho_p0_d;  // FP64 offsets and rho_f / rho_p for the initial fill
  double fr_d;
};

// Layout of the state inside the caller's buffer: np planes [ny][pitch] per time level.
struct Layout {
  int nx, ny, pitch;  // pitch: elements per row, rows 128-byte aligned
  size_t plane;       // elements per plane = pitch * ny
  int storage;        // MCLBM_STORE_F32, _F16 or _BF16
  int elem;           // bytes per element (4 or 2)
  int np;             // planes per time level: 27, or 36 with two thermal sets
};

struct StepArgs {
  const void* src;  // state level read (element type of L.storage)
  void* dst;        // state level written
  Layout L;
  int z_src;  // TMA kernel: first plane of the source level in the two-level tensor (0 or 27)
  int* err;   // device error word: bit 0 set when a bounded wait gave up
  uint32_t seed;             // 16-bit stochastic rounding: per-launch seed
  const uint32_t* epoch;     // 16-bit stochastic rounding: graph replay counter (device)
  StepConsts k;
};

// Host-side derivation (mclbm_model.cpp).
void props_default(mclbm_props* p);
int derive_consts(int nx, int ny, double Ra, double Pr, double phi, double d_p,
                  const mclbm_props& p, mclbm_consts* c);
StepConsts fold_step_consts(int nx, int ny, double phi, double d_p, const mclbm_props& p,
                            const mclbm_consts& c);

// Kernel launchers (mclbm_kernels.cu). All enqueue on `st` and return the launch error.
struct StepConfig {
  int variant;  // 0: tile kernel; 2: TMA-staged persistent tiles
  int grid;     // TMA kernel: persistent CTAs (set by prepare_step)
  bool sr;      // 16-bit storage: stochastic rounding (else round to nearest)
  int vec;      // nodes per thread of the step kernels: 1 or 2 (0: chosen by lattice size)
  bool two;     // FP32: pairs of steps by the two-step kernel (set by prepare_two_f32)
  int grid2;    // two-step kernel: CTAs (one per 32 x 16 tile)
  int th;       // TMA kernel: tile height, 8 or 7 (0 before prepare_step: chosen by lattice)
};
StepConfig choose_step_config(int nx, int ny, int np);
// Device-dependent set-up of the chosen variant (shared-memory limit, persistent grid size);
// may fall back to variant 0. Needs the device current.
cudaError_t prepare_step(StepConfig* c, const Layout& L);
// Tensor maps of the two-level state (x = column, y = row, z = plane of 54) for the TMA kernels
// with tiles tile_w x tile_h: maps[0] loads input windows (the tile with 16 bytes of columns and
// 2 rows of halo on each side), maps[1] stores output tiles.
cudaError_t make_state_tensor_map(CUtensorMap* maps, void* state0, const Layout& L, int tile_w,
                                  int tile_h);
// The two-step kernel's window loads (FP32): 32 x 16 tiles with 4 nodes of halo on each side.
cudaError_t make_two_step_tensor_map(CUtensorMap* map, void* state0, const Layout& L);
// Two-step kernel (FP32 storage): enables it in c when every SM can take one 32 x 16 tile
// (cudaErrorNotSupported otherwise); launches one two-step launch from a.src to a.dst.
cudaError_t prepare_two_f32(StepConfig* c, const Layout& L);
cudaError_t launch_two_f32(const StepArgs& a, const StepConfig& c, const CUtensorMap* map2,
                           cudaStream_t st);
// Tile width of a configured step kernel's TMA maps.
int step_tile_width(const StepConfig& c);
cudaError_t launch_step(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                        cudaStream_t st);
// Per storage type (mclbm_step_f32.cu, mclbm_step_f16.cu, mclbm_step_bf16.cu).
cudaError_t launch_step_f32(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                            cudaStream_t st);
cudaError_t launch_step_f16(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                            cudaStream_t st);
cudaError_t launch_step_bf16(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                             cudaStream_t st);
cudaError_t prepare_tma_f32(StepConfig* c, const Layout& L);
cudaError_t prepare_tma_f16(StepConfig* c, const Layout& L);
cudaError_t prepare_tma_bf16(StepConfig* c, const Layout& L);
// Advances the stochastic-rounding epoch by one (a single thread; captured after each graph).
cudaError_t launch_epoch_advance(uint32_t* epoch, cudaStream_t st);
cudaError_t launch_stream_only(const void* src, void* dst, const Layout& L, const StepConsts& k,
                               cudaStream_t st);
// warm: null (rest), [4][ny][nx] (ux, uy, theta, phi) or, with warm_rho, [5][ny][nx] (+ rho^w)
cudaError_t launch_init(void* dst, const Layout& L, const StepConsts& k, const float* warm,
                        int warm_rho, cudaStream_t st);
cudaError_t launch_fields(const void* src, const Layout& L, const StepConsts& k, uint32_t which,
                          float* out, cudaStream_t st);
// Nusselt partial sums: red[0] = sum_j (8 T_h - 9 th_0 + th_1) / 3, red[1] = cold-wall twin.
cudaError_t launch_nusselt(const void* src, const Layout& L, const StepConsts& k, double* red,
                           cudaStream_t st);
// Mass: red[0] = sum of f^w deviations, red[1] = sum of f^p deviations.
cudaError_t launch_mass(const void* src, const Layout& L, double* partials, double* red,
                        cudaStream_t st);
// Residual sums red[0..5] = |du|^2, |u|^2, dtheta^2, theta^2, dphi^2, phi^2 against snap;
// the snapshot [4][ny][nx] (ux, uy, theta, phi) is replaced.
cudaError_t launch_residual(const void* src, const Layout& L, const StepConsts& k, float* snap,
                            bool sums, double* partials, double* red, cudaStream_t st);
// to_packed: stored level -> packed FP32 deviations [np][ny][nx]; else the reverse.
cudaError_t launch_state_copy(const void* src, void* dst, const Layout& L, bool to_packed,
                              cudaStream_t st);

// ---- batched stepping of many cavities (mclbm_batch.cu) ------------------------------------
// One cavity of a batch as the batch kernel sees it (device memory, 64-byte aligned).
struct BatchCav {  // aligned like its CUtensorMap member
  CUtensorMap map;      // window loads of the cavity's two-level state
  CUtensorMap map_out;  // output tile stores (16-bit storage)
  void* level[2];   // the two state levels
  Layout L;
  StepConsts k;
  int cur;          // level that holds the state at batch creation (even step counts keep it)
};
struct BatchLaunch {
  const void* cavs;   // BatchCav[n]
  const void* tiles;  // tile table (cavity | tile column | tile row)
  int n_tiles;
  int grid;           // persistent CTAs
  int storage;
  bool sr, all_forces;
  const uint32_t* epoch;
  int* err;
};
cudaError_t launch_batch_step(const BatchLaunch& b, int parity, uint32_t seed, cudaStream_t st);
cudaError_t launch_batch_nusselt(const BatchLaunch& b, int n_cav, int parity, double* out,
                                 cudaStream_t st);
cudaError_t prepare_batch(int storage, int* per_sm);
void build_tile_table(const std::vector<int>& nx, const std::vector<int>& ny,
                      const std::vector<int>& active, int order, std::vector<uint32_t>* out);
constexpr int kBatchTileW = 64;  // batch tiles: 64 x 8 (two nodes per thread)
constexpr int kBatchTileH = 8;
int batch_size(const mclbm_batch_t* b);  // cavities of the batch (0 for NULL)

}  // namespace mcl
