// Internal definition of the libvlb context (shared by the API translation units).
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/vlb.h"
#include "vlb_launch.h"
#include "vlb_stage.cuh"
#include "vlb_channel.cuh"
#include "vlb_tables.h"

using namespace vlb;

struct vlb_ctx;
// Tile buffers and grid of a stage launch with the context's current launch shape
// over n_tiles tiles (the shape's configuration is computed once and kept).
cudaError_t stage_launch_config(vlb_ctx* c, int n_tiles, int* nbuf, int* grid);

struct vlb_ctx {
  int kind = 0;  // 0 circular Couette instances, 1 gradually expanding channel
  vlb_model model{};
  int prec = 0;
  int n_inst = 0;
  cudaStream_t stream = nullptr;
  AxisTables ax[2];
  int nq0 = 0, nq1 = 0, V = 0, Vp = 0;
  long long total_cells = 0;
  size_t esize = 8;
  std::vector<InstDesc> inst;
  std::vector<TileDesc> tiles;
  std::vector<GeoCell> geo;
  std::vector<vlb_couette_grid> grids;
  ModelArgs margs{};
  std::unique_ptr<KArgs<float>> k32;
  std::unique_ptr<KArgs<double>> k64;
  void* F[3] = {nullptr, nullptr, nullptr};
  StageVariant variants[16];
  int n_variants = 0;
  int variant = 0;
  // launch configuration per launch shape, computed on its first use (stage_launch_config)
  int cfg_nbuf[16] = {};
  int cfg_per_sm[16] = {};
  int sms = 0;  // SMs of the context's device
  int device = -1;  // CUDA device current when the context was created
  int cur = 0;   // buffer holding F_l
  int last = 0;  // buffer written by the most recent stage
  int stage_done = 0;
  InstDesc* d_inst = nullptr;
  TileDesc* d_tiles = nullptr;
  GeoCell* d_geo = nullptr;
  GeoCellF* d_geof = nullptr;
  double* d_nw = nullptr;
  WallEq* d_wall = nullptr;  // Couette: 2 per instance (inner, outer)
  unsigned* d_err = nullptr;
  double* d_mom = nullptr;
  double* d_prev = nullptr;
  double* d_res = nullptr;
  void* d_halo = nullptr;  // Couette: 2 x 3 ghost rows per instance for slab halo ends
  bool has_halo = false;   // some instance has a halo end (vlb_stage only)
  int collision = 0;       // vlb_collision: 0 BGK, 1 Shakhov
  // velocity sets beyond 32 nodes on an axis: the multi-kernel path of vlb_large.cu
  bool large = false;
  LargeModel lm{};
  void* d_lm = nullptr;      // the LargeModel tables (one allocation)
  double* d_lwall = nullptr;  // per (instance, wall): g0, g1, in_flux, T_w
  void* d_lrec = nullptr;     // per cell equilibrium record
  void* d_lforce = nullptr;   // per cell force term
  double* d_lpart = nullptr;  // per cell and wall chunk sums
  bool ftilde = false;        // the f~ formulation
  double* d_tgeo = nullptr;   // its per-cell geometry: sqrt(g), advp, advm, 1/R_s
  // f~ on the fused stage kernel (velocity sets of the fused path): launch shapes 0 and 1 only,
  // their own launch configurations, the geometry records (cp, cm = advp, advm; inv_rbar = 1/R_s),
  // sqrt(g) per cell and the inertial term of R per velocity in the bulk type
  bool ft_fused = false;
  int cfg_ft_nbuf[2] = {}, cfg_ft_per_sm[2] = {};
  GeoCell* d_ftgeo = nullptr;
  GeoCellF* d_ftgeof = nullptr;
  void* d_ftsg = nullptr;
  void* d_ftfr = nullptr;
  double prandtl = 1.0;
  bool have_prev = false;
  size_t tile_cap = 0;
  // channel
  ChanDesc cdesc{};
  ChanVariant cvariants[8];
  int n_cvariants = 0;
  ChanCell<double>* d_cgeo = nullptr;
  ChanCell<float>* d_cgeof = nullptr;
  CellMap cmap;  // device cell order against the caller's (identity for Couette)
  std::vector<unsigned char> chan_kp;  // ChanKP block (split force matrices), a kernel parameter
  void* d_ctab = nullptr;  // ChanTables of the model shape in the context's real type
  size_t ctab_bytes = 0;
  std::vector<double> chan_lc;    // lambda of the row centres
  double chan_phi_end[2] = {0, 0};  // phi at the inlet and outlet interfaces
  void* d_qflow = nullptr;        // flow-rate ends: 4 n_lambda reals (ChanArgs::qflow)
  double* d_cpost = nullptr;      // post-processing geometry: lambda_c, lambda_f, phi_c, phi'_c
  double* d_post = nullptr;       // post-processing outputs (allocated on first use)
  double chan_dxi = 0.0;
  vlb_channel_grid chan_grid{};   // the channel's grid parameters
  bool clb = false;               // the Cartesian-split formulation (Sec. VII.G) is on
  ClbGeom clbg{};                 // its geometry (device arrays in d_clbgeo)
  void* d_clbgeo = nullptr;
  // the Cartesian split on the marching channel kernel (shapes with a vielbein kernel): its
  // geometry records, read as described at channel_stage_kernel
  bool clb_march = false;
  ChanCell<double>* d_clbcgeo = nullptr;
  ChanCell<float>* d_clbcgeof = nullptr;
  void* d_clbrec = nullptr;       // per cell equilibrium record
  void* d_clbres = nullptr;       // per row and end: reservoir factors
  // CUDA graph of three RK3 steps (nine stage launches), replayed by vlb_step_graph
  // three-step graphs, one per starting buffer F[cur] (captured on first use)
  cudaGraphExec_t graph_exec[3] = {nullptr, nullptr, nullptr};
  cudaStream_t capture_stream = nullptr;
  int graph_variant[3] = {-1, -1, -1};
  long long launches = 0;
  long long steps = 0;
  std::string err;
};
