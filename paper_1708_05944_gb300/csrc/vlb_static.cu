// vlb_step_static_scratch: RK3 steps whose intermediate stage buffers live in a
// fixed device array compiled into the library, so the call allocates nothing.
//
// Who needs it: applications that cannot allocate device memory when they step
// -- their device memory belongs to another allocator or to a pool that is
// already full, or the call sits in a latency-critical loop where a
// cudaMalloc is not allowed.  They keep f in their own device buffers and
// call this entry point, which uses g_step_scratch below for F^(1) and F^(2).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <string>
#include <vector>

#include "vlb_ctx.h"

namespace {

// 64 MiB, held by every GPU that loads the library until the process exits.
constexpr size_t kScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_step_scratch[kScratchBytes];

// Device address of g_step_scratch per device, looked up on the first call
// made on that device (host threads may race to fill an entry; they store the
// same address).
constexpr int kMaxDevices = 64;
std::atomic<void*> g_scratch_ptr[kMaxDevices];

vlb_status static_fail(vlb_ctx* c, vlb_status s, const std::string& msg) {
  c->err = msg;
  return s;
}

template <typename real>
cudaError_t launch_one(vlb_ctx* c, int k, const void* prev, const void* fl, void* out) {
  StageArgs<real> a{};
  a.Fprev = static_cast<const real*>(prev);
  a.Fl = static_cast<const real*>(fl);
  a.Fout = static_cast<real*>(out);
  const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0}, cc[3] = {1.0, 0.25, 2.0 / 3.0};
  a.ca = ca[k - 1];
  a.cb = cb[k - 1];
  a.cc = cc[k - 1];
  a.caf = float(a.ca);
  a.cbf = float(a.cb);
  a.ccf = float(a.cc);
  a.inst = c->d_inst;
  a.tiles = c->d_tiles;
  a.n_tiles = int(c->tiles.size());
  a.geo = c->d_geo;
  a.geof = c->d_geof;
  a.nw = c->d_nw;
  a.wall = c->d_wall;
  a.err = c->d_err;
  a.Vp = c->Vp;
  a.max_polls = 1ull << 26;
  const KArgs<real>* kk;
  if constexpr (sizeof(real) == 4) kk = c->k32.get(); else kk = c->k64.get();
  int grid = 0;
  cudaError_t e = stage_launch_config(c, a.n_tiles, &a.nbuf, &grid);
  if (e != cudaSuccess) return e;
  return launch_stage<real>(c->variants[c->variant], a, c->margs, *kk, grid, c->stream);
}

}  // namespace

extern "C" vlb_status vlb_step_static_scratch(vlb_ctx* c, const void* f_in, void* f_out, double dt,
                                              long long nsteps) {
  if (!c) return VLB_ERR_INVALID;
  // Couette contexts only: the channel stage has its own kernel and buffers, and this
  // entry point launches nothing for it
  if (c->kind != 0) return static_fail(c, VLB_ERR_UNSUPPORTED, "static-scratch stepping covers Couette contexts only");
  if (c->has_halo) return static_fail(c, VLB_ERR_STATE, "a slab steps one stage at a time (vlb_stage)");
  if (c->collision != 0) return static_fail(c, VLB_ERR_UNSUPPORTED, "static-scratch stepping runs the BGK stage only");
  if (c->large || c->ftilde)
    return static_fail(c, VLB_ERR_UNSUPPORTED, "static-scratch stepping covers the chi formulation up to 32 nodes per axis");
  if (!f_in || !f_out || f_in == f_out) return static_fail(c, VLB_ERR_INVALID, "need distinct input and output buffers");
  if (nsteps < 1 || !(dt > 0.0) || !std::isfinite(dt))
    return static_fail(c, VLB_ERR_INVALID, "need a finite dt > 0 and nsteps >= 1");
  if (c->Vp != c->V)
    return static_fail(c, VLB_ERR_UNSUPPORTED, "velocity count must be a multiple of 4 for caller-owned buffers");
  const size_t fbytes = size_t(c->total_cells) * 2 * c->Vp * c->esize;
  if (2 * fbytes > kScratchBytes)
    return static_fail(c, VLB_ERR_UNSUPPORTED,
                       "two stage buffers of " + std::to_string(fbytes) + " bytes exceed the 64 MiB static scratch");
  // the array's address is per device: the context's device must be the current one
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_fail(c, VLB_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != c->device)
    return static_fail(c, VLB_ERR_INVALID, "the context's device must be the current device");
  if (dev < 0 || dev >= kMaxDevices) return static_fail(c, VLB_ERR_UNSUPPORTED, "device index out of range");
  void* addr = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!addr) {  // first call on this device: device address of the static array
    e = cudaGetSymbolAddress(&addr, g_step_scratch);
    if (e != cudaSuccess)
      return static_fail(c, VLB_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev].store(addr, std::memory_order_release);
  }
  unsigned char* base = static_cast<unsigned char*>(addr);
  void* s1 = base;
  void* s2 = base + fbytes;
  // time step for every instance: the same update as vlb_set_dt (a synchronising copy of the
  // instance descriptors), made only when dt differs from the context's current one
  bool change = false;
  for (int i = 0; i < c->n_inst; ++i) change |= c->inst[i].dt != dt;
  if (change) {
    std::vector<double> v(c->n_inst, dt);
    const vlb_status st = vlb_set_dt(c, v.data());
    if (st != VLB_OK) return st;
  }
  // the stage kernels work on the deviation D = F - R from the rest state: convert f_in into
  // f_out, step f_out (stage 3 updates it in place: each CTA reads only its own F_l rows), and
  // convert f_out back at the end
  e = c->prec == VLB_FP64
          ? launch_deviation<double>(static_cast<const double*>(f_in), static_cast<double*>(f_out), c->total_cells,
                                     c->Vp, c->margs, 1, c->stream)
          : launch_deviation<float>(static_cast<const float*>(f_in), static_cast<float*>(f_out), c->total_cells,
                                    c->Vp, c->margs, 1, c->stream);
  if (e != cudaSuccess) return static_fail(c, VLB_ERR_CUDA, std::string("conversion launch: ") + cudaGetErrorString(e));
  for (long long s = 0; s < nsteps; ++s) {
    const void* Fl = f_out;
    for (int k = 1; k <= 3; ++k) {
      const void* prev = k == 1 ? Fl : (k == 2 ? s1 : s2);
      void* out = k == 1 ? s1 : (k == 2 ? s2 : f_out);
      e = c->prec == VLB_FP64 ? launch_one<double>(c, k, prev, Fl, out) : launch_one<float>(c, k, prev, Fl, out);
      if (e != cudaSuccess) return static_fail(c, VLB_ERR_CUDA, std::string("stage launch: ") + cudaGetErrorString(e));
    }
  }
  e = c->prec == VLB_FP64
          ? launch_deviation<double>(static_cast<const double*>(f_out), static_cast<double*>(f_out), c->total_cells,
                                     c->Vp, c->margs, 0, c->stream)
          : launch_deviation<float>(static_cast<const float*>(f_out), static_cast<float*>(f_out), c->total_cells,
                                    c->Vp, c->margs, 0, c->stream);
  if (e != cudaSuccess) return static_fail(c, VLB_ERR_CUDA, std::string("conversion launch: ") + cudaGetErrorString(e));
  return VLB_OK;
}
