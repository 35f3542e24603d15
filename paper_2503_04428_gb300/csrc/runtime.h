// runtime.h -- host-side context of a handle (shared by the C-ABI translation units).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/hydro.h"
#include "common.cuh"

namespace hydro {

void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define HCK(call)                                        \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

struct DeviceArena {
  std::vector<void*> ptrs;
  int alloc(void** p, size_t bytes);
  void release();
};

struct BatchState;  // batched-tube extension (api_batch.cu)

}  // namespace hydro

// Internal entry points shared between the C-ABI translation units.
int hydro_common_init(hydro_ctx* h, int precision, void* stream);
int hydro_batch_set_state_impl(hydro_ctx* h, const void* U, int where);
int hydro_batch_get_state_impl(hydro_ctx* h, void* U, int where);
int hydro_batch_stats_impl(hydro_ctx* h, hydro_stats_t* out);
void hydro_batch_free_impl(hydro_ctx* h);
namespace hydro {
template <typename T> Gas<T> make_gas(double gm);
template <typename T> GasRad<T> make_gas_rad(double gm, double R, double a);
int tune_cache_get(const std::string& key, int* value, double* us);
void tune_cache_put(const std::string& key, int value, double us);
std::string device_key();
}  // namespace hydro

struct hydro_ctx {
  bool batched = false;
  int precision = 64;
  size_t esize = 8;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  int device = 0;
  int num_sms = 0;
  // grid
  int dim = 1, n[3] = {1, 1, 1}, coords = 0, riemann = 1, limiter = 1, ns = 0, nsx = 0, nv = 3;
  int bc[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  double gamma = 1.4;
  int eos_rad = 0;                   // 1: gas + radiation EoS (Eq. 6-7)
  double R_gas = 0.0, a_rad = 0.0;   // its constants
  double eps_dual = 0.0;             // dual-energy criterion (Sect. 2.5); 0 = off
  long long ncell = 0;
  std::vector<double> faces[3];
  void* buf[2] = {nullptr, nullptr};
  hydro::Ctrl* ctrl = nullptr;       // device control block
  hydro::Ctrl* ctrl_host = nullptr;  // pinned mirror
  void* geo[32] = {nullptr};         // device geometry arrays (precision T)
  double* dvol[3] = {nullptr, nullptr, nullptr};  // FP64 volume factors a, b, c
  float* dvz32 = nullptr;            // c as FP32 pairs (hi, lo), hi + lo = c to ~2^-48 (FP32 in-step totals)
  double* rc_d = nullptr;            // FP64 radial centres
  double omega = 4.0 * 3.14159265358979323846;
  // sources
  int gravity = 0, heating = 0;
  double g0[3] = {0, 0, 0}, G = 0, Mc = 0, heat_prm[4] = {0, 0, 0, 0};
  void* gmono = nullptr;
  double* shell = nullptr;
  double* shell_partial = nullptr;
  int shell_kchunk = 1, shell_nchunks = 1;
  // totals
  double* tot_partial = nullptr;
  double* tot_out = nullptr;
  int tot_blocks = 0;
  // totals accumulated in the step: on, valid for the current state, the
  // per-CTA partials [nv][ctas]
  bool step_tot = false, step_tot_ok = false;
  double* step_tot_part = nullptr;
  // launch shape
  int zchunk = 32;
  int tile_x = 0, tile_y = 0, threads = 0;
  double tuned_us = 0.0;
  bool tuned = false;
  // domain decomposition (Sect. 3.3.1): exchanged sides of axis xaxis, the
  // two face coordinates beyond each (nearest first), their halo buffers
  // [nv][2][cross section] on the device, and the monopole's inner mass
  int xaxis = -1;
  bool xch[2] = {false, false};
  double xg[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  void* halo_d[2] = {nullptr, nullptr};
  void* pack_d = nullptr;    // staging of hydro_get_boundary for host output
  double inner_mass = 0.0;
  // moving grid (Sect. 3.1.1): axis, face velocity, volume ratios (device)
  int maxis = -1;
  double wgrid = 0.0;
  void* vr_d = nullptr;
  void* irn_d = nullptr;  // 1/r of the radial cells after the step
  // graph of one device-dt step
  cudaGraphExec_t graph = nullptr;
  double graph_cfl = -1.0, graph_tend = -2.0;
  long long faces_per_step = 0;
  long long steps_host = 0;
  hydro::DeviceArena arena;
  hydro::BatchState* bs = nullptr;
};
