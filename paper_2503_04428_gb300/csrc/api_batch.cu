// api_batch.cu -- C ABI of the batched-tube form, the MLP guess network and
// the standalone exact Riemann solver (include/hydro.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "batched.cuh"
#include "mlp.cuh"
#include "runtime.h"

namespace hydro {

// Autotuner candidates: warps per CTA, cells per work item (whole 28-cell
// segments) and persistent CTAs per SM (up to the occupancy limit).
static const int BATCH_NW[] = {4, 8};
static const int BATCH_ITEM[] = {28, 56, 112, 224, 448, 896, 1792, 2800, 3584, 4200, 5376, 8204};  // 8204 >= the longest tube
// Steps per launch that the autotuner times (one launch runs any number of
// steps; several let it see the steps overlap).
static const int TUNE_STEPS = 6;

struct BatchState {
  int ntubes = 0;
  long long total = 0;
  long long stride = 0;  // device elements between the variables' slabs: total rounded up to 16 bytes
  long long faces_per_step = 0;
  long long* off_d = nullptr;
  std::vector<long long> off;
  // per tube (see BatchArgs): speed slots (3 x ntubes); items completed in
  // the running launch and the launch step of the last dt added, side by
  // side (2 x ntubes words, zeroed before every launch by one memset); time
  // and time before the last dt
  unsigned long long* smax = nullptr;
  unsigned int* tcnt = nullptr;
  double* t_tube = nullptr;
  double* t_prev = nullptr;
  BatchCtrl* bctrl = nullptr;
  BatchCtrl* bctrl_host = nullptr;
  // launch shape: warps per CTA, cells per item, CTAs
  int nw = 8, item_len = 112, grid = 0;
  BatchItem* items = nullptr;  // one step's work items in tube order (device)
  int nitems = 0;
  std::vector<int> item_first;  // first item of every tube (+ end)
  std::vector<BatchItem> h_items;  // the items (host)
  // host-resident runs: per-part control blocks, copy streams and events
  int nparts = 0;
  BatchCtrl* part_ctrl = nullptr;
  BatchCtrl* part_ctrl_host = nullptr;
  cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_done;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // the host-resident run as a CUDA graph, for repeated calls on the same
  // pinned buffers
  cudaGraphExec_t host_graph = nullptr;
  // captured step launches (counter reset + one launch of n steps), by
  // (n, cfl); a few are kept
  std::vector<std::pair<std::pair<int, double>, cudaGraphExec_t>> step_graphs;
  int hg_parts = 0, hg_nsteps = 0;
  const void* hg_in = nullptr;
  void* hg_out = nullptr;
  double hg_cfl = -1.0;
  // MLP
  float* w = nullptr;
  MlpSmemW* w_packed = nullptr;  // w in the batched kernel's shared-memory layout
  float* m = nullptr;
  float* v = nullptr;
  bool w_set = false;
  int mlp_on = 0;
  // harvesting
  double* harvest = nullptr;
  unsigned long long* harvest_n = nullptr;
  long long harvest_cap = 0;
  unsigned long long harvest_thresh = 0, harvest_seed = 0;
  bool tuned = false;
  double tuned_us = 0.0;
  int limiter = 1;
};

static int berr(const std::string& m) {
  set_error(m);
  return HYDRO_ERR_ARG;
}

// Allow the ring's dynamic shared memory (once per instantiation and device).
template <typename T, int NW>
static int batch_attr() {
  HCK(smem_attr_once((const void*)batched_kernel<T, NW>, (int)batched_smem_bytes<T, NW>()));
  return HYDRO_OK;
}

template <typename T, int NW>
static int launch_batch_nw(hydro_ctx* h, const BatchArgs<T>& a, int grid) {
  int st = batch_attr<T, NW>();
  if (st) return st;
  batched_kernel<T, NW><<<grid, NW * 32, batched_smem_bytes<T, NW>(), h->stream>>>(a);
  HCK(cudaGetLastError());
  return HYDRO_OK;
}

template <typename T>
static int occupancy_nw(int nw, int* blocks) {
  int st = nw == 4 ? batch_attr<T, 4>() : batch_attr<T, 8>();
  if (st) return st;
  if (nw == 4)
    HCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batched_kernel<T, 4>, 128, batched_smem_bytes<T, 4>()));
  else
    HCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batched_kernel<T, 8>, 256, batched_smem_bytes<T, 8>()));
  return HYDRO_OK;
}

static void drop_graph(BatchState* bs);

static int upload_items(const std::vector<BatchItem>& items, BatchItem** d_items) {
  cudaFree(*d_items);
  *d_items = nullptr;
  HCK(cudaMalloc(d_items, sizeof(BatchItem) * std::max<size_t>(1, items.size())));
  HCK(cudaMemcpy(*d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
  return HYDRO_OK;
}

// Work items of item_len cells (the last of a tube shorter), in tube order:
// every step of a launch hands them out in this order, so a tube's items of
// the next step come a whole step of the other tubes' items after its own
// (the items of a group of consecutive tubes are one contiguous range).
static int make_items(hydro_ctx* h, int item_len) {
  BatchState* bs = h->bs;
  bs->h_items.clear();
  bs->item_first.assign(bs->ntubes + 1, 0);
  for (int b = 0; b < bs->ntubes; ++b) {
    bs->item_first[b] = (int)bs->h_items.size();
    const int nb = (int)(bs->off[b + 1] - bs->off[b]);
    const int nit = (nb + item_len - 1) / item_len;
    for (int s0 = 0; s0 < nb; s0 += item_len) {
      BatchItem it;
      std::memset(&it, 0, sizeof(it));
      it.base = bs->off[b];
      it.nb = nb;
      it.beg = s0;
      it.end = std::min(s0 + item_len, nb);
      it.tube = b;
      it.nit = nit;
      bs->h_items.push_back(it);
    }
  }
  bs->item_first[bs->ntubes] = (int)bs->h_items.size();
  bs->item_len = item_len;
  bs->nitems = (int)bs->h_items.size();
  drop_graph(bs);
  return upload_items(bs->h_items, &bs->items);
}

// Per-tube bookkeeping arrays of one run (the handle's, or the autotuner's
// scratch copies).
struct TubeArrays {
  unsigned long long* smax;  // 3 x ntubes
  unsigned int* tcnt;        // 2 x ntubes: item counts, then launch steps (tstart)
  double* t_tube;
  double* t_prev;
};

static TubeArrays tube_arrays(const BatchState* bs) { return {bs->smax, bs->tcnt, bs->t_tube, bs->t_prev}; }

template <typename T>
static BatchArgs<T> batch_args(hydro_ctx* h, double cfl, BatchCtrl* ctrl, const TubeArrays& ta, int nsteps) {
  BatchState* bs = h->bs;
  BatchArgs<T> a;
  a.A = (const T*)h->buf[0];
  a.Aw = (T*)h->buf[0];
  a.B = (T*)h->buf[1];
  a.stride = bs->stride;
  a.items = bs->items;
  a.nitems = bs->nitems;
  a.nsteps = nsteps;
  a.ntot = bs->ntubes;
  a.smax = ta.smax;
  a.tcnt = ta.tcnt;
  a.tstart = reinterpret_cast<int*>(ta.tcnt + bs->ntubes);
  a.t_tube = ta.t_tube;
  a.t_prev = ta.t_prev;
  a.cfl = cfl;
  a.gas = make_gas<T>(h->gamma);
  a.limiter = bs->limiter;
  a.mlp_w = bs->w_packed;
  a.mlp_on = bs->mlp_on && bs->w_set;
  a.harvest = bs->harvest;
  a.harvest_n = bs->harvest_n;
  a.harvest_cap = bs->harvest_cap;
  a.harvest_thresh = bs->harvest_thresh;
  a.harvest_seed = bs->harvest_seed;
  a.ctrl = ctrl;
  return a;
}

template <typename T>
static int launch_batch_a(hydro_ctx* h, const BatchArgs<T>& a) {
  if (h->bs->nw == 4) return launch_batch_nw<T, 4>(h, a, h->bs->grid);
  return launch_batch_nw<T, 8>(h, a, h->bs->grid);
}

// One launch of nsteps steps of every tube (on the handle's buffers), after
// clearing the per-launch item counts.
static int launch_batch(hydro_ctx* h, double cfl, BatchCtrl* ctrl, const TubeArrays& ta, int nsteps) {
  if (nsteps < 1) return HYDRO_OK;
  HCK(cudaMemsetAsync(ta.tcnt, 0, sizeof(unsigned int) * 2 * h->bs->ntubes, h->stream));
  return h->precision == 64 ? launch_batch_a<double>(h, batch_args<double>(h, cfl, ctrl, ta, nsteps))
                            : launch_batch_a<float>(h, batch_args<float>(h, cfl, ctrl, ta, nsteps));
}

static int read_bctrl(hydro_ctx* h) {
  HCK(cudaMemcpyAsync(h->bs->bctrl_host, h->bs->bctrl, sizeof(BatchCtrl), cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

static int write_bctrl(hydro_ctx* h) {
  HCK(cudaMemcpyAsync(h->bs->bctrl, h->bs->bctrl_host, sizeof(BatchCtrl), cudaMemcpyHostToDevice, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

static void drop_graph(BatchState* bs) {
  if (bs->host_graph) {
    cudaGraphExecDestroy(bs->host_graph);
    bs->host_graph = nullptr;
  }
  for (auto& g : bs->step_graphs) cudaGraphExecDestroy(g.second);
  bs->step_graphs.clear();
}

// Autotuner of the batched launch: warps per CTA, cells per work item and
// persistent CTAs per SM, each candidate timed with CUDA events on a launch
// of TUNE_STEPS steps from the current state, run on scratch copies of the
// state, the per-tube arrays and the control block (the handle's state is
// untouched).
// Share of the current state's interior faces whose two cells differ: 0
// (below a quarter), 1 (below three quarters) or 2.  The best launch shape
// depends on it (long work items pay where most cells take the uniform
// shortcut, short ones where every face runs the solver), so it is part of
// the autotuner's cache key.
static int state_roughness(hydro_ctx* h, int* cls) {
  BatchState* bs = h->bs;
  int st = read_bctrl(h);
  if (st) return st;
  unsigned long long* d = nullptr;
  HCK(cudaMalloc(&d, sizeof(unsigned long long)));
  HCK(cudaMemsetAsync(d, 0, sizeof(unsigned long long), h->stream));
  if (h->precision == 64)
    batch_rough_kernel<double><<<bs->ntubes, 256, 0, h->stream>>>((const double*)h->buf[bs->bctrl_host->c.cur],
                                                                   bs->stride, bs->off_d, d);
  else
    batch_rough_kernel<float><<<bs->ntubes, 256, 0, h->stream>>>((const float*)h->buf[bs->bctrl_host->c.cur],
                                                                  bs->stride, bs->off_d, d);
  HCK(cudaGetLastError());
  unsigned long long c = 0;
  HCK(cudaMemcpyAsync(&c, d, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  cudaFree(d);
  const double f = (double)c / (double)std::max<long long>(1, bs->total - bs->ntubes);
  *cls = f < 0.25 ? 0 : (f < 0.75 ? 1 : 2);
  return HYDRO_OK;
}

static int autotune_batch(hydro_ctx* h, double cfl) {
  BatchState* bs = h->bs;
  if (bs->tuned) return HYDRO_OK;
  bs->tuned = true;
  int rough = 0;
  int st0 = state_roughness(h, &rough);
  if (st0) return st0;
  std::ostringstream key;
  key << "batchms_p" << h->precision << "_t" << bs->ntubes << "_c" << bs->total << "_m" << bs->mlp_on << "_r"
      << rough << "_" << device_key();
  int cached;
  double us;
  if (tune_cache_get(key.str(), &cached, &us)) {
    // cached = (warps * 10000 + item cells) * 100 + CTAs per SM
    bs->nw = cached / 1000000;
    bs->grid = h->num_sms * (cached % 100);
    int st = make_items(h, (cached / 100) % 10000);
    if (st) return st;
    bs->tuned_us = us;
    return HYDRO_OK;
  }
  int st = read_bctrl(h);
  if (st) return st;
  const int n = bs->ntubes;
  const size_t sbytes = (size_t)3 * bs->stride * h->esize;
  BatchCtrl base = *bs->bctrl_host;
  const int cur = base.c.cur;
  base.c.status = 0;
  base.c.done = 0;
  base.c.cur = 0;
  base.next_entry = 0;
  BatchCtrl* sc = nullptr;
  TubeArrays sa = {nullptr, nullptr, nullptr, nullptr};
  void* sbuf[2] = {nullptr, nullptr};
  void* const hbuf[2] = {h->buf[0], h->buf[1]};
  auto release = [&]() {
    cudaStreamSynchronize(h->stream);
    h->buf[0] = hbuf[0];
    h->buf[1] = hbuf[1];
    cudaFree(sc);
    cudaFree(sa.smax);
    cudaFree(sa.tcnt);
    cudaFree(sa.t_tube);
    cudaFree(sa.t_prev);
    cudaFree(sbuf[0]);
    cudaFree(sbuf[1]);
  };
  if (cudaMalloc(&sc, sizeof(BatchCtrl)) || cudaMalloc(&sa.smax, sizeof(unsigned long long) * 3 * n) ||
      cudaMalloc(&sa.tcnt, sizeof(unsigned int) * 2 * n) || cudaMalloc(&sa.t_tube, sizeof(double) * n) ||
      cudaMalloc(&sa.t_prev, sizeof(double) * n) || cudaMalloc(&sbuf[0], sbytes) || cudaMalloc(&sbuf[1], sbytes)) {
    release();
    set_error("hydro_batch_run: autotuner scratch allocation failed");
    return HYDRO_ERR_OOM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300;
  int best_nw = 8, best_item = 3584, best_mult = 1;
  auto reset = [&]() {
    cudaMemcpyAsync(sc, &base, sizeof(BatchCtrl), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(sbuf[0], hbuf[cur], sbytes, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(sa.smax, bs->smax, sizeof(unsigned long long) * 3 * n, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemsetAsync(sa.t_tube, 0, sizeof(double) * n, h->stream);
  };
  h->buf[0] = sbuf[0];
  h->buf[1] = sbuf[1];
  for (int nw : BATCH_NW) {
    bs->nw = nw;
    int occ = 1;
    st = h->precision == 64 ? occupancy_nw<double>(nw, &occ) : occupancy_nw<float>(nw, &occ);
    if (st) break;
    for (int item : BATCH_ITEM) {
      for (int mult = 1; mult <= std::max(1, occ); ++mult) {
        bs->grid = h->num_sms * mult;
        if ((st = make_items(h, item))) break;
        const int reps = 2;
        float ms = 0.f;
        reset();
        if ((st = launch_batch(h, cfl, sc, sa, TUNE_STEPS))) break;
        for (int r = 0; r < reps; ++r) {
          reset();
          cudaEventRecord(e0, h->stream);
          if ((st = launch_batch(h, cfl, sc, sa, TUNE_STEPS))) break;
          cudaEventRecord(e1, h->stream);
          cudaEventSynchronize(e1);
          float m1 = 0.f;
          cudaEventElapsedTime(&m1, e0, e1);
          ms += m1;
        }
        if (st) break;
        const double t = 1000.0 * ms / (reps * TUNE_STEPS);
        if (t < best) {
          best = t;
          best_nw = nw;
          best_item = item;
          best_mult = mult;
        }
      }
      if (st) break;
    }
    if (st) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release();
  if (st) return st;
  bs->nw = best_nw;
  bs->grid = h->num_sms * best_mult;
  if ((st = make_items(h, best_item))) return st;
  bs->tuned_us = best;
  tune_cache_put(key.str(), (best_nw * 10000 + best_item) * 100 + best_mult, best);
  return HYDRO_OK;
}

// The per-tube bookkeeping of the state in buffer `slot` (speeds, step
// counts, times 0; see batch_init_kernel) and its validity (*status).
template <typename T>
static int batch_init(hydro_ctx* h, int slot, int* status) {
  BatchState* bs = h->bs;
  int* d_status = nullptr;
  HCK(cudaMalloc(&d_status, sizeof(int)));
  HCK(cudaMemsetAsync(d_status, 0, sizeof(int), h->stream));
  batch_init_kernel<T><<<bs->ntubes, 256, 0, h->stream>>>((const T*)h->buf[slot], bs->stride, bs->off_d, 0,
                                                           bs->ntubes, make_gas<T>(h->gamma), &bs->bctrl->c,
                                                           bs->ntubes, bs->smax, bs->tcnt,
                                                           reinterpret_cast<int*>(bs->tcnt + bs->ntubes),
                                                           bs->t_tube, bs->t_prev, d_status);
  HCK(cudaGetLastError());
  HCK(cudaMemcpyAsync(status, d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  cudaFree(d_status);
  return HYDRO_OK;
}

// After a failed launch: every tube's last good state into buffer `cur` of
// the launch's start, the bookkeeping restarted at its step count s0 (see
// batch_settle_kernel).
template <typename T>
static int batch_settle(hydro_ctx* h, long long s0, int cur) {
  BatchState* bs = h->bs;
  batch_settle_kernel<T><<<bs->ntubes, 256, 0, h->stream>>>(
      (T*)h->buf[0], (T*)h->buf[1], bs->stride, bs->off_d, bs->item_len, make_gas<T>(h->gamma), s0, cur,
      bs->ntubes, bs->smax, bs->tcnt, reinterpret_cast<int*>(bs->tcnt + bs->ntubes), bs->t_tube, bs->t_prev);
  HCK(cudaGetLastError());
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

// Glorot-uniform initial weights from SplitMix64 (zero biases).
static void init_weights(std::vector<float>& w, unsigned long long seed) {
  w.assign(MLP_NPARAM, 0.f);
  unsigned long long state = seed;
  auto next = [&]() {
    state += 0x9E3779B97F4A7C15ull;
    unsigned long long z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](int off, int n, int fan_in, int fan_out) {
    const double a = std::sqrt(6.0 / (fan_in + fan_out));
    for (int i = 0; i < n; ++i) w[off + i] = (float)(a * (2.0 * next() - 1.0));
  };
  fill(MW1, MLP_H * MLP_IN, MLP_IN, MLP_H);
  fill(MW2, MLP_H * MLP_H, MLP_H, MLP_H);
  fill(MW3, MLP_H, MLP_H, 1);
}

static int ensure_mlp(hydro_ctx* h) {
  BatchState* bs = h->bs;
  if (!bs->w) {
    HCK(cudaMalloc(&bs->w_packed, sizeof(MlpSmemW)));
    HCK(cudaMalloc(&bs->w, sizeof(float) * MLP_NPARAM));
    HCK(cudaMalloc(&bs->m, sizeof(float) * MLP_NPARAM));
    HCK(cudaMalloc(&bs->v, sizeof(float) * MLP_NPARAM));
  }
  return HYDRO_OK;
}

// The kernel's copy of the weights, after every change of bs->w.
static int pack_mlp(hydro_ctx* h) {
  mlp_pack_kernel<<<1, 256, 0, h->stream>>>(h->bs->w, h->bs->w_packed);
  HCK(cudaGetLastError());
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

// Gradient of the MSE over `count` samples (rows idx[first..] of X/Y) into grad.
static int mlp_gradient(cudaStream_t s, const float* W, const float* X, const float* Y, const int* idx,
                        long long first, long long count, float* partial, double* loss_partial,
                        double* grad, double* loss_acc) {
  HCK(smem_attr_once((const void*)mlp_grad_kernel, (int)sizeof(MlpSmem)));
  const int nblocks = (int)((count + MLP_SB - 1) / MLP_SB);
  mlp_grad_kernel<<<nblocks, 256, sizeof(MlpSmem), s>>>(W, X, Y, idx, first, count, (float)(1.0 / count),
                                                        partial, loss_partial);
  HCK(cudaGetLastError());
  mlp_reduce_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(partial, nblocks, grad, loss_partial, loss_acc);
  HCK(cudaGetLastError());
  return HYDRO_OK;
}

// A wait that cannot complete: thread 0 arms an mbarrier for 16 bytes that no
// copy delivers (none is issued) and waits on it with the batched kernel's
// bounded wait (mbar_wait), which must give up and report a timeout.
__global__ void wait_probe_kernel(int* status) {
  __shared__ unsigned long long bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  mbar_expect_tx(&bar, 16u);
  *status = mbar_wait(&bar, 0u) ? HYDRO_OK : ST_TIMEOUT;
}

}  // namespace hydro

using namespace hydro;

int hydro_batch_set_state_impl(hydro_ctx* h, const void* U, int where) {
  BatchState* bs = h->bs;
  int st = read_bctrl(h);
  if (st) return st;
  const int slot = bs->bctrl_host->c.cur ^ 1;
  // caller layout: 3 slabs of total elements; device: slabs `stride` apart
  HCK(cudaMemcpy2DAsync(h->buf[slot], (size_t)bs->stride * h->esize, U, (size_t)bs->total * h->esize,
                        (size_t)bs->total * h->esize, 3,
                        where == HYDRO_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  // the speeds of the new state go to the slots of the current step count
  // (the rest of the bookkeeping is written only if the state is valid)
  std::vector<unsigned long long> keep_smax(3 * (size_t)bs->ntubes);
  std::vector<double> keep_t(2 * (size_t)bs->ntubes);
  HCK(cudaMemcpyAsync(keep_smax.data(), bs->smax, sizeof(unsigned long long) * 3 * bs->ntubes,
                      cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaMemcpyAsync(keep_t.data(), bs->t_tube, sizeof(double) * bs->ntubes, cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaMemcpyAsync(keep_t.data() + bs->ntubes, bs->t_prev, sizeof(double) * bs->ntubes, cudaMemcpyDeviceToHost,
                      h->stream));
  int status = 0;
  st = h->precision == 64 ? batch_init<double>(h, slot, &status) : batch_init<float>(h, slot, &status);
  if (st) return st;
  if (status) {
    // the previous state and its bookkeeping stay
    HCK(cudaMemcpyAsync(bs->smax, keep_smax.data(), sizeof(unsigned long long) * 3 * bs->ntubes,
                        cudaMemcpyHostToDevice, h->stream));
    HCK(cudaMemcpyAsync(bs->t_tube, keep_t.data(), sizeof(double) * bs->ntubes, cudaMemcpyHostToDevice,
                        h->stream));
    HCK(cudaMemcpyAsync(bs->t_prev, keep_t.data() + bs->ntubes, sizeof(double) * bs->ntubes,
                        cudaMemcpyHostToDevice, h->stream));
    HCK(cudaStreamSynchronize(h->stream));
    set_error(status == HYDRO_ERR_NONFINITE ? "hydro_set_state: non-finite value in the state"
                                            : "hydro_set_state: density or pressure not positive");
    return status;
  }
  bs->bctrl_host->c.cur = slot;
  bs->bctrl_host->c.status = 0;
  bs->bctrl_host->c.done = 0;
  bs->bctrl_host->c.err_step = -1;
  bs->bctrl_host->next_entry = 0;
  return write_bctrl(h);
}

int hydro_batch_get_state_impl(hydro_ctx* h, void* U, int where) {
  int st = read_bctrl(h);
  if (st) return st;
  const BatchState* bs = h->bs;
  HCK(cudaMemcpy2DAsync(U, (size_t)bs->total * h->esize, h->buf[bs->bctrl_host->c.cur], (size_t)bs->stride * h->esize,
                        (size_t)bs->total * h->esize, 3,
                        where == HYDRO_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

int hydro_batch_stats_impl(hydro_ctx* h, hydro_stats_t* out) {
  int st = read_bctrl(h);
  if (st) return st;
  const Ctrl& c = h->bs->bctrl_host->c;
  std::memset(out, 0, sizeof(*out));
  out->steps = c.step;
  out->faces = c.step * h->bs->faces_per_step;
  out->newton_iters = (long long)c.iters;
  out->fallbacks = (long long)c.fallbacks;
  out->mlp_faces = (long long)c.mlp;
  for (int k = 0; k < NCAT; ++k) {
    out->newton_faces[k] = (long long)h->bs->bctrl_host->cat_faces[k];
    out->newton_iters_by[k] = (long long)h->bs->bctrl_host->cat_iters[k];
  }
  out->tile_x = h->bs->item_len;
  out->tile_y = h->bs->nw;
  out->zchunk = h->bs->grid;
  out->threads = h->bs->nw * 32;
  out->tuned_us_per_step = h->bs->tuned_us;
  return HYDRO_OK;
}

void hydro_batch_free_impl(hydro_ctx* h) {
  BatchState* bs = h->bs;
  drop_graph(bs);
  cudaFree(bs->part_ctrl);
  cudaFreeHost(bs->part_ctrl_host);
  if (bs->ev_fork) cudaEventDestroy(bs->ev_fork);
  if (bs->ev_join) cudaEventDestroy(bs->ev_join);
  if (bs->s_h2d) cudaStreamDestroy(bs->s_h2d);
  if (bs->s_d2h) cudaStreamDestroy(bs->s_d2h);
  for (cudaEvent_t e : bs->ev_in) cudaEventDestroy(e);
  for (cudaEvent_t e : bs->ev_done) cudaEventDestroy(e);
  cudaFree(bs->off_d);
  cudaFree(bs->smax);
  cudaFree(bs->tcnt);
  cudaFree(bs->t_tube);
  cudaFree(bs->t_prev);
  cudaFree(bs->bctrl);
  cudaFreeHost(bs->bctrl_host);
  cudaFree(bs->items);
  cudaFree(bs->w);
  cudaFree(bs->w_packed);
  cudaFree(bs->m);
  cudaFree(bs->v);
  cudaFree(bs->harvest);
  cudaFree(bs->harvest_n);
  delete bs;
  h->bs = nullptr;
}

// Pipelined host-resident run: the tubes are split into parts of about equal
// cell counts; part p's input copy (stream s_h2d), its steps (the handle's
// stream) and its output copy (stream s_d2h) are ordered by events, so the
// copies of one part overlap the computation of others.  Every part has its
// own control block and work-queue range; the per-cell arithmetic is that of
// hydro_batch_set_state + hydro_batch_run + hydro_batch_get_state.
// Every device operation of one host-resident run, on the handle's stream
// with the two copy streams forked from and joined back to it (so that the
// sequence can be captured as one graph): the parts' control blocks in, then
// per part the input copy, speeds and validity, the steps and the output
// copy, and the control blocks back out.
template <typename T>
static int enqueue_host_run(hydro_ctx* h, const T* U_in, T* U_out, int nsteps, double cfl, int P,
                            const std::vector<int>& b0) {
  BatchState* bs = h->bs;
  int st = HYDRO_OK;
  const int slot = 0, out_slot = nsteps & 1;
  const Gas<T> gas = make_gas<T>(h->gamma);
  T* buf_in = (T*)h->buf[slot];
  T* buf_out = (T*)h->buf[out_slot];
  HCK(cudaMemcpyAsync(bs->part_ctrl, bs->part_ctrl_host, sizeof(BatchCtrl) * P, cudaMemcpyHostToDevice, h->stream));
  HCK(cudaEventRecord(bs->ev_fork, h->stream));
  HCK(cudaStreamWaitEvent(bs->s_h2d, bs->ev_fork, 0));
  HCK(cudaStreamWaitEvent(bs->s_d2h, bs->ev_fork, 0));
  for (int p = 0; p < P; ++p) {
    const int t0 = b0[p], t1 = b0[p + 1];
    if (t1 <= t0) continue;
    const long long c0 = bs->off[t0], nc = bs->off[t1] - c0;
    // the group's cells of the three variables in one strided copy (measured
    // ~4 % faster than three copies for the whole pattern)
    HCK(cudaMemcpy2DAsync(buf_in + c0, sizeof(T) * bs->stride, U_in + c0, sizeof(T) * bs->total, sizeof(T) * nc, 3,
                          cudaMemcpyHostToDevice, bs->s_h2d));
    HCK(cudaEventRecord(bs->ev_in[p], bs->s_h2d));
    HCK(cudaStreamWaitEvent(h->stream, bs->ev_in[p], 0));
    // the part's per-tube speeds, step counts, times and validity (as
    // hydro_batch_set_state), in one kernel: no copy-engine work between the
    // part's input and its steps
    batch_init_kernel<T><<<t1 - t0, 256, 0, h->stream>>>(buf_in, bs->stride, bs->off_d, t0, t1 - t0, gas,
                                                        &bs->part_ctrl[p].c, bs->ntubes, bs->smax, bs->tcnt,
                                                        reinterpret_cast<int*>(bs->tcnt + bs->ntubes), bs->t_tube,
                                                        bs->t_prev, &bs->part_ctrl[p].c.status);
    HCK(cudaGetLastError());
    // the part's steps in one launch over its tubes' items
    BatchArgs<T> a = batch_args<T>(h, cfl, &bs->part_ctrl[p], tube_arrays(bs), nsteps);
    const int i0 = bs->item_first[t0], i1 = bs->item_first[t1];
    a.items = bs->items + i0;
    a.nitems = i1 - i0;
    if ((st = launch_batch_a<T>(h, a))) return st;
    HCK(cudaEventRecord(bs->ev_done[p], h->stream));
    HCK(cudaStreamWaitEvent(bs->s_d2h, bs->ev_done[p], 0));
    HCK(cudaMemcpy2DAsync(U_out + c0, sizeof(T) * bs->total, buf_out + c0, sizeof(T) * bs->stride, sizeof(T) * nc, 3,
                          cudaMemcpyDeviceToHost, bs->s_d2h));
  }
  HCK(cudaMemcpyAsync(bs->part_ctrl_host, bs->part_ctrl, sizeof(BatchCtrl) * P, cudaMemcpyDeviceToHost,
                      h->stream));
  HCK(cudaEventRecord(bs->ev_join, bs->s_d2h));
  HCK(cudaStreamWaitEvent(h->stream, bs->ev_join, 0));
  return st;
}

template <typename T>
static int batch_run_host_t(hydro_ctx* h, const T* U_in, T* U_out, int nsteps, double cfl, int nparts) {
  BatchState* bs = h->bs;
  const int P = std::max(1, std::min(nparts, bs->ntubes));
  if (bs->nparts < P) {
    drop_graph(bs);  // the host-run graph refers to the old control blocks
    cudaFree(bs->part_ctrl);
    cudaFreeHost(bs->part_ctrl_host);
    bs->part_ctrl = nullptr;
    bs->part_ctrl_host = nullptr;
    bs->nparts = 0;
    HCK(cudaMalloc(&bs->part_ctrl, sizeof(BatchCtrl) * P));
    HCK(cudaMallocHost(&bs->part_ctrl_host, sizeof(BatchCtrl) * P));
    bs->nparts = P;
  }
  if (!bs->s_h2d) HCK(cudaStreamCreateWithFlags(&bs->s_h2d, cudaStreamNonBlocking));
  if (!bs->s_d2h) HCK(cudaStreamCreateWithFlags(&bs->s_d2h, cudaStreamNonBlocking));
  if (!bs->ev_fork) HCK(cudaEventCreateWithFlags(&bs->ev_fork, cudaEventDisableTiming));
  if (!bs->ev_join) HCK(cudaEventCreateWithFlags(&bs->ev_join, cudaEventDisableTiming));
  while ((int)bs->ev_in.size() < P) {
    cudaEvent_t a, b;
    HCK(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    HCK(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    bs->ev_in.push_back(a);
    bs->ev_done.push_back(b);
  }
  int st = read_bctrl(h);
  if (st) return st;
  // part boundaries at tubes, about total/P cells each
  std::vector<int> b0(P + 1, bs->ntubes);
  b0[0] = 0;
  for (int p = 1, b = 0; p < P; ++p) {
    const long long target = bs->total * p / P;
    while (b < bs->ntubes && bs->off[b] < target) ++b;
    b0[p] = std::max(b, b0[p - 1] + 1);
  }
  for (int p = 1; p <= P; ++p) b0[p] = std::min(std::max(b0[p], b0[p - 1]), bs->ntubes);
  b0[P] = bs->ntubes;
  const int slot = 0;  // input lands in buffer 0; the result is in buffer (nsteps & 1)
  const int out_slot = nsteps & 1;
  for (int p = 0; p < P; ++p) {
    BatchCtrl& c = bs->part_ctrl_host[p];
    std::memset(&c, 0, sizeof(BatchCtrl));
    c.c.cur = slot;
    c.c.step = bs->bctrl_host->c.step;
    c.c.err_step = -1;
  }
  // Reuse the captured graph for the same buffers and settings; capture one
  // for pinned buffers; enqueue directly otherwise (a graph cannot hold
  // copies from pageable memory).
  const bool same = bs->host_graph && bs->hg_parts == P && bs->hg_nsteps == nsteps && bs->hg_in == U_in &&
                    bs->hg_out == U_out && bs->hg_cfl == cfl;
  if (!same) {
    if (bs->host_graph) {
      cudaGraphExecDestroy(bs->host_graph);
      bs->host_graph = nullptr;
    }
    cudaPointerAttributes ai, ao;
    const bool pinned = cudaPointerGetAttributes(&ai, U_in) == cudaSuccess && ai.type == cudaMemoryTypeHost &&
                        cudaPointerGetAttributes(&ao, U_out) == cudaSuccess && ao.type == cudaMemoryTypeHost;
    cudaGetLastError();  // an unregistered pointer may leave an error behind
    if (pinned) {
      cudaGraph_t g;
      HCK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed));
      st = enqueue_host_run<T>(h, U_in, U_out, nsteps, cfl, P, b0);
      cudaError_t e = cudaStreamEndCapture(h->stream, &g);
      if (st) {
        if (e == cudaSuccess) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(e, "hydro_batch_run_host: cudaStreamEndCapture");
      e = cudaGraphInstantiate(&bs->host_graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "hydro_batch_run_host: cudaGraphInstantiate");
      bs->hg_parts = P;
      bs->hg_nsteps = nsteps;
      bs->hg_in = U_in;
      bs->hg_out = U_out;
      bs->hg_cfl = cfl;
    } else {
      if ((st = enqueue_host_run<T>(h, U_in, U_out, nsteps, cfl, P, b0))) return st;
    }
  }
  if (bs->host_graph) HCK(cudaGraphLaunch(bs->host_graph, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  int code = 0;
  long long iters = 0, mlp = 0, fb = 0;
  unsigned long long cf[NCAT] = {0, 0, 0}, ci[NCAT] = {0, 0, 0};
  for (int p = 0; p < P; ++p) {
    const Ctrl& c = bs->part_ctrl_host[p].c;
    if (c.status && !code) code = c.status;
    iters += (long long)c.iters;
    mlp += (long long)c.mlp;
    fb += (long long)c.fallbacks;
    for (int k = 0; k < NCAT; ++k) {
      cf[k] += bs->part_ctrl_host[p].cat_faces[k];
      ci[k] += bs->part_ctrl_host[p].cat_iters[k];
    }
  }
  // the handle now holds the result, as after set_state + run
  BatchCtrl& g = *bs->bctrl_host;
  g.c.status = 0;
  g.c.done = 0;
  g.c.err_step = -1;
  g.next_entry = 0;
  if (!code) {
    g.c.cur = out_slot;
    g.c.step += nsteps;
    g.c.iters += iters;
    g.c.mlp += mlp;
    g.c.fallbacks += fb;
    for (int k = 0; k < NCAT; ++k) {
      g.cat_faces[k] += cf[k];
      g.cat_iters[k] += ci[k];
    }
  }
  if ((st = write_bctrl(h))) return st;
  if (code) {
    // consistent bookkeeping for whatever the current buffer now holds
    int ignored = 0;
    if ((st = batch_init<T>(h, g.c.cur, &ignored))) return st;
    set_error("hydro_batch_run_host: device status " + std::to_string(code) +
              " (the state copied in is invalid or a step failed); the output is unspecified");
    return code;
  }
  return HYDRO_OK;
}

extern "C" {

int hydro_wait_probe(double* seconds_out) {
  int* d_status = nullptr;
  HCK(cudaMalloc(&d_status, sizeof(int)));
  cudaEvent_t e0, e1;
  HCK(cudaEventCreate(&e0));
  HCK(cudaEventCreate(&e1));
  HCK(cudaEventRecord(e0, 0));
  wait_probe_kernel<<<1, 32>>>(d_status);
  HCK(cudaGetLastError());
  HCK(cudaEventRecord(e1, 0));
  HCK(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  int status = HYDRO_ERR_CUDA;
  HCK(cudaMemcpy(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_status);
  if (seconds_out) *seconds_out = 1e-3 * ms;
  if (status == ST_TIMEOUT) set_error("hydro_wait_probe: the bounded wait expired (the expected outcome)");
  return status;
}

int hydro_batch_create(const int* lengths, int ntubes, const hydro_eos* eos, int riemann, int limiter,
                       int precision, void* stream, hydro_t* out) {
  if (!lengths || !eos || !out || ntubes < 1) return berr("hydro_batch_create: bad argument");
  *out = nullptr;
  if (riemann != HYDRO_EXACT)
    return set_error("hydro_batch_create: the batched form uses the exact Riemann solver"), HYDRO_ERR_UNSUPPORTED;
  if (eos->n_scalars != 0) return berr("hydro_batch_create: tubes carry no passive scalars");
  if (!(eos->gamma > 1.0)) return berr("hydro_batch_create: gamma must exceed 1");
  if (limiter < HYDRO_FIRST_ORDER || limiter > HYDRO_VANALBADA) return berr("hydro_batch_create: bad limiter");
  long long total = 0;
  for (int b = 0; b < ntubes; ++b) {
    if (lengths[b] < 2) return berr("hydro_batch_create: every tube needs >= 2 cells");
    total += lengths[b];
  }
  if (total > 0x7fffffffLL) return berr("hydro_batch_create: more than 2^31 cells in total");
  hydro_ctx* h = new hydro_ctx();
  h->batched = true;
  int st = hydro_common_init(h, precision, stream);
  if (st) { hydro_destroy(h); return st; }
  h->gamma = eos->gamma;
  h->riemann = riemann;
  h->limiter = limiter;
  h->dim = 1;
  h->nv = 3;
  h->ncell = total;
  BatchState* bs = new BatchState();
  h->bs = bs;
  bs->ntubes = ntubes;
  bs->total = total;
  const long long q = 16 / h->esize;
  bs->stride = (total + q - 1) / q * q;
  bs->limiter = limiter;
  bs->faces_per_step = total + ntubes;
  bs->off.assign(ntubes + 1, 0);
  for (int b = 0; b < ntubes; ++b) bs->off[b + 1] = bs->off[b] + lengths[b];
  const size_t bytes = (size_t)3 * bs->stride * h->esize;
  for (int b = 0; b < 2; ++b)
    if ((st = h->arena.alloc(&h->buf[b], bytes))) { hydro_destroy(h); return st; }
  if (cudaMalloc(&bs->off_d, sizeof(long long) * (ntubes + 1)) != cudaSuccess ||
      cudaMalloc(&bs->smax, sizeof(unsigned long long) * 3 * ntubes) != cudaSuccess ||
      cudaMalloc(&bs->tcnt, sizeof(unsigned int) * 2 * ntubes) != cudaSuccess ||
      cudaMalloc(&bs->t_tube, sizeof(double) * ntubes) != cudaSuccess ||
      cudaMalloc(&bs->t_prev, sizeof(double) * ntubes) != cudaSuccess ||
      cudaMalloc(&bs->bctrl, sizeof(BatchCtrl)) != cudaSuccess ||
      cudaMallocHost(&bs->bctrl_host, sizeof(BatchCtrl)) != cudaSuccess) {
    set_error("hydro_batch_create: device allocation failed");
    hydro_destroy(h);
    return HYDRO_ERR_OOM;
  }
  cudaMemcpy(bs->off_d, bs->off.data(), sizeof(long long) * (ntubes + 1), cudaMemcpyHostToDevice);
  cudaMemset(bs->smax, 0, sizeof(unsigned long long) * 3 * ntubes);
  cudaMemset(bs->tcnt, 0, sizeof(unsigned int) * 2 * ntubes);
  cudaMemset(bs->t_tube, 0, sizeof(double) * ntubes);
  cudaMemset(bs->t_prev, 0, sizeof(double) * ntubes);
  std::memset(bs->bctrl_host, 0, sizeof(BatchCtrl));
  bs->bctrl_host->c.err_step = -1;
  if ((st = write_bctrl(h)) || (st = make_items(h, 112))) { hydro_destroy(h); return st; }
  bs->grid = h->num_sms * 2;
  *out = h;
  return HYDRO_OK;
}

int hydro_batch_run_host(hydro_t h, const void* U_in, void* U_out, int nsteps, double cfl, int nparts) {
  if (!h || !h->batched || !U_in || !U_out) return berr("hydro_batch_run_host: bad argument");
  if (nsteps < 1 || !(cfl > 0.0)) return berr("hydro_batch_run_host: need nsteps >= 1 and cfl > 0");
  if (nparts < 0) return berr("hydro_batch_run_host: nparts must be >= 0");
  int st;
  if ((st = autotune_batch(h, cfl))) return st;
  if (nparts == 0) nparts = 8;
  return h->precision == 64
             ? batch_run_host_t<double>(h, (const double*)U_in, (double*)U_out, nsteps, cfl, nparts)
             : batch_run_host_t<float>(h, (const float*)U_in, (float*)U_out, nsteps, cfl, nparts);
}

int hydro_batch_enqueue(hydro_t h, int nsteps, double cfl) {
  if (!h || !h->batched) return berr("hydro_batch_enqueue: batched handle required");
  if (nsteps < 0 || !(cfl > 0.0)) return berr("hydro_batch_enqueue: bad nsteps or cfl");
  BatchState* bs = h->bs;
  int st;
  if ((st = autotune_batch(h, cfl))) return st;
  if (nsteps == 0) return HYDRO_OK;
  // all the steps in one launch (no grid-wide barrier between them),
  // replayed from a captured graph of that launch
  cudaGraphExec_t ge = nullptr;
  for (auto& g : bs->step_graphs)
    if (g.first.first == nsteps && g.first.second == cfl) ge = g.second;
  if (!ge) {
    if (bs->step_graphs.size() >= 16) {
      for (auto& g : bs->step_graphs) cudaGraphExecDestroy(g.second);
      bs->step_graphs.clear();
    }
    // the kernel's shared-memory limit is raised before the capture
    if ((st = h->precision == 64 ? (bs->nw == 4 ? batch_attr<double, 4>() : batch_attr<double, 8>())
                                 : (bs->nw == 4 ? batch_attr<float, 4>() : batch_attr<float, 8>())))
      return st;
    cudaGraph_t g;
    HCK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed));
    st = launch_batch(h, cfl, bs->bctrl, tube_arrays(bs), nsteps);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (st) {
      if (e == cudaSuccess) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "hydro_batch_enqueue: cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "hydro_batch_enqueue: cudaGraphInstantiate");
    bs->step_graphs.push_back({{nsteps, cfl}, ge});
  }
  HCK(cudaGraphLaunch(ge, h->stream));
  return HYDRO_OK;
}

int hydro_batch_run(hydro_t h, int nsteps, double cfl) {
  if (!h || !h->batched) return berr("hydro_batch_run: batched handle required");
  if (nsteps < 0 || !(cfl > 0.0)) return berr("hydro_batch_run: bad nsteps or cfl");
  BatchState* bs = h->bs;
  int st;
  if ((st = hydro_batch_enqueue(h, nsteps, cfl))) return st;
  if ((st = read_bctrl(h))) return st;
  const int code = bs->bctrl_host->c.status;
  if (code == 0) return HYDRO_OK;
  std::ostringstream m;
  m << "hydro_batch_run: device status " << code << " at step " << bs->bctrl_host->c.err_step;
  // the failed launch left step and buffer as at its start: every tube's
  // last good state back into that buffer
  st = h->precision == 64 ? batch_settle<double>(h, bs->bctrl_host->c.step, bs->bctrl_host->c.cur)
                          : batch_settle<float>(h, bs->bctrl_host->c.step, bs->bctrl_host->c.cur);
  if (st) return st;
  bs->bctrl_host->c.status = 0;
  bs->bctrl_host->c.done = 0;
  bs->bctrl_host->c.err_step = -1;
  bs->bctrl_host->next_entry = 0;
  if ((st = write_bctrl(h))) return st;
  set_error(m.str());
  return code;
}

int hydro_harvest_begin(hydro_t h, long capacity, double keep_prob, unsigned long long seed) {
  if (!h || !h->batched || capacity < 0 || !(keep_prob >= 0.0 && keep_prob <= 1.0))
    return berr("hydro_harvest_begin: bad argument");
  BatchState* bs = h->bs;
  cudaFree(bs->harvest);
  cudaFree(bs->harvest_n);
  bs->harvest = nullptr;
  bs->harvest_n = nullptr;
  bs->harvest_cap = capacity;
  if (capacity > 0) {
    HCK(cudaMalloc(&bs->harvest, sizeof(double) * 6 * capacity));
    HCK(cudaMalloc(&bs->harvest_n, sizeof(unsigned long long)));
    HCK(cudaMemset(bs->harvest_n, 0, sizeof(unsigned long long)));
  }
  bs->harvest_thresh = keep_prob >= 1.0 ? ~0ull : (unsigned long long)(keep_prob * 18446744073709551616.0);
  bs->harvest_seed = seed;
  drop_graph(bs);
  return HYDRO_OK;
}

int hydro_harvest_get(hydro_t h, double* faces6, long cap, long* n) {
  if (!h || !h->batched || !n) return berr("hydro_harvest_get: bad argument");
  BatchState* bs = h->bs;
  *n = 0;
  if (!bs->harvest) return HYDRO_OK;
  unsigned long long cnt = 0;
  HCK(cudaStreamSynchronize(h->stream));
  HCK(cudaMemcpy(&cnt, bs->harvest_n, sizeof(cnt), cudaMemcpyDeviceToHost));
  long long m = std::min<long long>((long long)cnt, bs->harvest_cap);
  m = std::min<long long>(m, cap);
  if (m > 0 && faces6) HCK(cudaMemcpy(faces6, bs->harvest, sizeof(double) * 6 * m, cudaMemcpyDeviceToHost));
  *n = (long)m;
  return HYDRO_OK;
}

int hydro_mlp_set(hydro_t h, const float* weights, int enable) {
  if (!h || !h->batched) return berr("hydro_mlp_set: batched handle required");
  BatchState* bs = h->bs;
  int st = ensure_mlp(h);
  if (st) return st;
  if (weights) {
    HCK(cudaMemcpy(bs->w, weights, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice));
    if ((st = pack_mlp(h))) return st;
    bs->w_set = true;
  }
  if (enable && !bs->w_set) return berr("hydro_mlp_set: no weights to enable");
  bs->mlp_on = enable ? 1 : 0;
  drop_graph(bs);
  bs->tuned = bs->tuned && true;
  return HYDRO_OK;
}

int hydro_mlp_get(hydro_t h, float* weights_out) {
  if (!h || !h->batched || !weights_out) return berr("hydro_mlp_get: bad argument");
  if (!h->bs->w_set) return berr("hydro_mlp_get: the network has no weights yet");
  HCK(cudaMemcpy(weights_out, h->bs->w, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost));
  return HYDRO_OK;
}

int hydro_mlp_train(hydro_t h, const double* faces6, const double* log_pstar, long n, int epochs, int batch,
                    float lr, unsigned long long seed, double* loss_out) {
  if (!h || !h->batched || !faces6 || !log_pstar || n < 1 || epochs < 0 || batch < 1 || !(lr > 0.f))
    return berr("hydro_mlp_train: bad argument");
  BatchState* bs = h->bs;
  int st = ensure_mlp(h);
  if (st) return st;
  if (!bs->w_set) {
    std::vector<float> w0;
    init_weights(w0, seed);
    HCK(cudaMemcpy(bs->w, w0.data(), sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice));
    if ((st = pack_mlp(h))) return st;
    bs->w_set = true;
  }
  HCK(cudaMemset(bs->m, 0, sizeof(float) * MLP_NPARAM));
  HCK(cudaMemset(bs->v, 0, sizeof(float) * MLP_NPARAM));
  const long long bsz = std::min<long long>(batch, n);
  const int nblocks = (int)((bsz + MLP_SB - 1) / MLP_SB);
  double *f6 = nullptr, *lp = nullptr, *grad = nullptr, *lpart = nullptr, *lacc = nullptr;
  float *X = nullptr, *Y = nullptr, *part = nullptr;
  int* idx = nullptr;
  cudaStream_t s = h->stream;
  auto cleanup = [&]() {
    cudaFree(f6); cudaFree(lp); cudaFree(grad); cudaFree(lpart); cudaFree(lacc);
    cudaFree(X); cudaFree(Y); cudaFree(part); cudaFree(idx);
  };
  if (cudaMalloc(&f6, sizeof(double) * 6 * n) || cudaMalloc(&lp, sizeof(double) * n) ||
      cudaMalloc(&X, sizeof(float) * 6 * n) || cudaMalloc(&Y, sizeof(float) * n) ||
      cudaMalloc(&idx, sizeof(int) * n) || cudaMalloc(&part, sizeof(float) * MLP_NPARAM * nblocks) ||
      cudaMalloc(&lpart, sizeof(double) * nblocks) || cudaMalloc(&grad, sizeof(double) * MLP_NPARAM) ||
      cudaMalloc(&lacc, sizeof(double))) {
    cleanup();
    set_error("hydro_mlp_train: device allocation failed");
    return HYDRO_ERR_OOM;
  }
  unsigned char* use_d = nullptr;
  if (cudaMalloc(&use_d, n)) {
    cleanup();
    set_error("hydro_mlp_train: device allocation failed");
    return HYDRO_ERR_OOM;
  }
  cudaMemcpyAsync(f6, faces6, sizeof(double) * 6 * n, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(lp, log_pstar, sizeof(double) * n, cudaMemcpyHostToDevice, s);
  mlp_features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f6, lp, n, make_gas<double>(h->gamma), X, Y,
                                                                  use_d);
  // train on the faces where the network is used (two-shock Toro estimate)
  std::vector<unsigned char> use(n);
  cudaMemcpyAsync(use.data(), use_d, n, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  cudaFree(use_d);
  std::vector<int> rows;
  for (long i = 0; i < n; ++i)
    if (use[i]) rows.push_back((int)i);
  if (rows.empty()) {
    cleanup();
    return berr("hydro_mlp_train: no sample passes the network's gate (two-shock Toro estimate, pressure jump > 4)");
  }
  const long m_use = (long)rows.size();
  const long long bsz_use = std::min<long long>(bsz, m_use);
  const long long steps_per_epoch = m_use / bsz_use;
  const long long total_steps = steps_per_epoch * (long long)epochs;
  std::vector<int> perm(m_use);
  HCK(smem_attr_once((const void*)mlp_grad_kernel, (int)sizeof(MlpSmem)));
  unsigned long long state = seed ^ 0xD1B54A32D192ED03ull;
  auto next = [&]() {
    state += 0x9E3779B97F4A7C15ull;
    unsigned long long z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  int step = 0;
  double loss = 0.0;
  for (int ep = 0; ep < epochs && st == 0; ++ep) {
    for (long i = 0; i < m_use; ++i) perm[i] = rows[i];
    for (long i = m_use - 1; i > 0; --i) std::swap(perm[i], perm[next() % (unsigned long long)(i + 1)]);
    cudaMemcpyAsync(idx, perm.data(), sizeof(int) * m_use, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(lacc, 0, sizeof(double), s);
    for (long long first = 0; first + bsz_use <= m_use; first += bsz_use) {
      // cosine decay of the learning rate over the whole run
      const double lr_t = 0.5 * (double)lr * (1.0 + std::cos(3.14159265358979323846 * step / (double)total_steps));
      ++step;
      const int nblk = (int)((bsz_use + MLP_SB - 1) / MLP_SB);
      mlp_grad_kernel<<<nblk, 256, sizeof(MlpSmem), s>>>(bs->w, X, Y, idx, first, bsz_use,
                                                         (float)(1.0 / bsz_use), part, lpart);
      mlp_reduce_adam_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(part, nblk, lpart, lacc, bs->w, bs->m,
                                                                      bs->v, step, lr_t, 0.9, 0.999, 1e-8);
      if (cudaGetLastError() != cudaSuccess) { st = HYDRO_ERR_CUDA; break; }
    }
    cudaMemcpyAsync(&loss, lacc, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    loss /= (double)(steps_per_epoch * bsz_use);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cleanup();
  if (st) return st;
  if (e != cudaSuccess) return cuda_fail(e, "hydro_mlp_train");
  if ((st = pack_mlp(h))) return st;
  if (loss_out) *loss_out = loss;
  drop_graph(bs);
  return HYDRO_OK;
}

int hydro_mlp_loss_grad(const float* weights, const double* x6, const double* target, long n, double* grad_out,
                        double* loss_out) {
  if (!weights || !x6 || !target || n < 1 || !grad_out) return berr("hydro_mlp_loss_grad: bad argument");
  std::vector<float> xf(6 * n), yf(n);
  for (long i = 0; i < 6 * n; ++i) xf[i] = (float)x6[i];
  for (long i = 0; i < n; ++i) yf[i] = (float)target[i];
  const int nblocks = (int)((n + MLP_SB - 1) / MLP_SB);
  float *W = nullptr, *X = nullptr, *Y = nullptr, *part = nullptr;
  double *grad = nullptr, *lpart = nullptr, *lacc = nullptr;
  HCK(cudaMalloc(&W, sizeof(float) * MLP_NPARAM));
  HCK(cudaMalloc(&X, sizeof(float) * 6 * n));
  HCK(cudaMalloc(&Y, sizeof(float) * n));
  HCK(cudaMalloc(&part, sizeof(float) * MLP_NPARAM * nblocks));
  HCK(cudaMalloc(&grad, sizeof(double) * MLP_NPARAM));
  HCK(cudaMalloc(&lpart, sizeof(double) * nblocks));
  HCK(cudaMalloc(&lacc, sizeof(double)));
  HCK(cudaMemcpy(W, weights, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice));
  HCK(cudaMemcpy(X, xf.data(), sizeof(float) * 6 * n, cudaMemcpyHostToDevice));
  HCK(cudaMemcpy(Y, yf.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
  HCK(cudaMemset(lacc, 0, sizeof(double)));
  int st = mlp_gradient(0, W, X, Y, nullptr, 0, n, part, lpart, grad, lacc);
  double loss = 0.0;
  if (!st) {
    HCK(cudaMemcpy(grad_out, grad, sizeof(double) * MLP_NPARAM, cudaMemcpyDeviceToHost));
    HCK(cudaMemcpy(&loss, lacc, sizeof(double), cudaMemcpyDeviceToHost));
  }
  cudaFree(W); cudaFree(X); cudaFree(Y); cudaFree(part); cudaFree(grad); cudaFree(lpart); cudaFree(lacc);
  if (loss_out) *loss_out = loss / n;
  return st;
}

int hydro_exact_solve(const double* WL, const double* WR, long n, double gamma, int guess, const float* weights,
                      int precision, double* pstar, double* ustar, int* iters) {
  if (!WL || !WR || n < 1 || !pstar || !ustar || !iters || !(gamma > 1.0))
    return berr("hydro_exact_solve: bad argument");
  if (precision != 32 && precision != 64) return berr("hydro_exact_solve: precision must be 32 or 64");
  if (guess == HYDRO_GUESS_MLP && !weights) return berr("hydro_exact_solve: MLP guess needs weights");
  double *dl = nullptr, *dr = nullptr, *dp = nullptr, *du = nullptr;
  int* di = nullptr;
  float* dw = nullptr;
  HCK(cudaMalloc(&dl, sizeof(double) * 3 * n));
  HCK(cudaMalloc(&dr, sizeof(double) * 3 * n));
  HCK(cudaMalloc(&dp, sizeof(double) * n));
  HCK(cudaMalloc(&du, sizeof(double) * n));
  HCK(cudaMalloc(&di, sizeof(int) * n));
  HCK(cudaMemcpy(dl, WL, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
  HCK(cudaMemcpy(dr, WR, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
  if (guess == HYDRO_GUESS_MLP) {
    HCK(cudaMalloc(&dw, sizeof(float) * MLP_NPARAM));
    HCK(cudaMemcpy(dw, weights, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice));
  }
  const unsigned blocks = (unsigned)((n + 127) / 128);
  if (precision == 64)
    exact_list_kernel<double><<<blocks, 128>>>(dl, dr, n, make_gas<double>(gamma), dw, dp, du, di);
  else
    exact_list_kernel<float><<<blocks, 128>>>(dl, dr, n, make_gas<float>(gamma), dw, dp, du, di);
  HCK(cudaGetLastError());
  HCK(cudaMemcpy(pstar, dp, sizeof(double) * n, cudaMemcpyDeviceToHost));
  HCK(cudaMemcpy(ustar, du, sizeof(double) * n, cudaMemcpyDeviceToHost));
  HCK(cudaMemcpy(iters, di, sizeof(int) * n, cudaMemcpyDeviceToHost));
  cudaFree(dl); cudaFree(dr); cudaFree(dp); cudaFree(du); cudaFree(di); cudaFree(dw);
  return HYDRO_OK;
}

int hydro_exact_sample(const double* WL, const double* WR, long nf, double gamma, const long long* face_of,
                       const double* xi, long npts, double* W_out) {
  if (!WL || !WR || nf < 1 || npts < 0 || (npts > 0 && (!face_of || !xi || !W_out)) || !(gamma > 1.0))
    return berr("hydro_exact_sample: bad argument");
  for (long k = 0; k < npts; ++k)
    if (face_of[k] < 0 || face_of[k] >= nf || !std::isfinite(xi[k]))
      return berr("hydro_exact_sample: face index out of range or non-finite x/t");
  if (npts == 0) return HYDRO_OK;
  double *dl = nullptr, *dr = nullptr, *dp = nullptr, *du = nullptr, *dxi = nullptr, *dw = nullptr;
  long long* df = nullptr;
  int* di = nullptr;
  auto cleanup = [&]() {
    cudaFree(dl); cudaFree(dr); cudaFree(dp); cudaFree(du); cudaFree(dxi); cudaFree(dw);
    cudaFree(df); cudaFree(di);
  };
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) { if (e == cudaSuccess) e = r; return e == cudaSuccess; };
  ok(cudaMalloc(&dl, sizeof(double) * 3 * nf)) && ok(cudaMalloc(&dr, sizeof(double) * 3 * nf)) &&
      ok(cudaMalloc(&dp, sizeof(double) * nf)) && ok(cudaMalloc(&du, sizeof(double) * nf)) &&
      ok(cudaMalloc(&di, sizeof(int) * nf)) && ok(cudaMalloc(&df, sizeof(long long) * npts)) &&
      ok(cudaMalloc(&dxi, sizeof(double) * npts)) && ok(cudaMalloc(&dw, sizeof(double) * 3 * npts)) &&
      ok(cudaMemcpy(dl, WL, sizeof(double) * 3 * nf, cudaMemcpyHostToDevice)) &&
      ok(cudaMemcpy(dr, WR, sizeof(double) * 3 * nf, cudaMemcpyHostToDevice)) &&
      ok(cudaMemcpy(df, face_of, sizeof(long long) * npts, cudaMemcpyHostToDevice)) &&
      ok(cudaMemcpy(dxi, xi, sizeof(double) * npts, cudaMemcpyHostToDevice));
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "hydro_exact_sample");
  }
  const Gas<double> gas = make_gas<double>(gamma);
  exact_list_kernel<double><<<(unsigned)((nf + 127) / 128), 128>>>(dl, dr, nf, gas, nullptr, dp, du, di);
  std::vector<double> ps(nf);
  ok(cudaGetLastError()) && ok(cudaMemcpy(ps.data(), dp, sizeof(double) * nf, cudaMemcpyDeviceToHost));
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "hydro_exact_sample");
  }
  for (long f = 0; f < nf; ++f)
    if (!(ps[f] > 0.0)) {
      cleanup();
      set_error("hydro_exact_sample: no star state (vacuum or Newton failure) at face " + std::to_string(f));
      return HYDRO_ERR_NEWTON;
    }
  exact_sample_kernel<<<(unsigned)((npts + 255) / 256), 256>>>(dl, dr, dp, du, df, dxi, npts, gas, dw);
  ok(cudaGetLastError()) && ok(cudaMemcpy(W_out, dw, sizeof(double) * 3 * npts, cudaMemcpyDeviceToHost));
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "hydro_exact_sample");
  return HYDRO_OK;
}

int hydro_batch_set_launch(hydro_t h, int warps_per_cta, int item_cells, int ctas_per_sm) {
  if (!h || !h->batched) return berr("hydro_batch_set_launch: batched handle required");
  if (warps_per_cta != 4 && warps_per_cta != 8) return berr("hydro_batch_set_launch: 4 or 8 warps per CTA");
  if (item_cells < BSEG || item_cells % BSEG != 0 || item_cells > 9999)
    return berr("hydro_batch_set_launch: item_cells must be a multiple of 28 in [28, 9996]");
  int occ = 1;
  int st = h->precision == 64 ? occupancy_nw<double>(warps_per_cta, &occ) : occupancy_nw<float>(warps_per_cta, &occ);
  if (st) return st;
  if (ctas_per_sm < 1 || ctas_per_sm > std::max(1, occ))
    return berr("hydro_batch_set_launch: ctas_per_sm must be in [1, " + std::to_string(std::max(1, occ)) + "]");
  BatchState* bs = h->bs;
  bs->nw = warps_per_cta;
  bs->grid = h->num_sms * ctas_per_sm;
  if ((st = make_items(h, item_cells))) return st;
  bs->tuned = true;
  bs->tuned_us = 0.0;
  return HYDRO_OK;
}

int hydro_batch_times(hydro_t h, double* t_out) {
  if (!h || !h->batched || !t_out) return berr("hydro_batch_times: bad argument");
  HCK(cudaMemcpyAsync(t_out, h->bs->t_tube, sizeof(double) * h->bs->ntubes, cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Gradient of the guess network without device allocation.
//
// hydro_mlp_loss_grad_device is for callers that cannot allocate device
// memory while they call in: code running inside CUDA stream capture, memory
// managed entirely by a host framework's own pool, or a process that must not
// grow its device footprint.  Its per-CTA partial gradients live in the
// file-scope array below instead of in cudaMalloc'd scratch.
// ---------------------------------------------------------------------------
namespace hydro {

constexpr long NOALLOC_MAX_SAMPLES = 16384;                    // n limit of one call
constexpr int NOALLOC_MAX_BLOCKS = (int)(NOALLOC_MAX_SAMPLES / MLP_SB);  // 256 CTAs
constexpr size_t NOALLOC_GRAD_BYTES = (size_t)NOALLOC_MAX_BLOCKS * MLP_NPARAM * sizeof(float);
constexpr size_t NOALLOC_BYTES = NOALLOC_GRAD_BYTES + (size_t)NOALLOC_MAX_BLOCKS * sizeof(double);

// 4.79 MB, held by every GPU that loads the library until the process exits.
// Every call reuses it: each CTA first writes all of its partial values and
// the reduction reads only the partials of the current call, so nothing has
// to be cleared between calls; calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Per-device set-up, done once per device with that device current and under
// one lock: the array's device address (the host-side symbol is only a
// stand-in and must not be passed to a kernel) and the gradient kernel's
// raised shared-memory limit, which is a per-device property of the kernel.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};
static bool g_noalloc_attr[64] = {false};

static int noalloc_scratch(void** out) {
  int dev = 0;
  HCK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("hydro_mlp_loss_grad_device: device index out of range");
    return HYDRO_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = p;
  }
  if (!g_noalloc_attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(MlpSmem));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(mlp_grad_kernel)");
    g_noalloc_attr[dev] = true;
  }
  *out = g_noalloc_ptr[dev];
  return HYDRO_OK;
}

// grad[p] = sum of the partials of parameter p (fixed order, FP64);
// loss = sum of the loss partials / n.
__global__ void noalloc_reduce_kernel(const float* partial, const double* loss_partial, int nblocks, long n,
                                      double* grad, double* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < MLP_NPARAM) {
    double a = 0.0;
    for (int b = 0; b < nblocks; ++b) a += (double)partial[(long long)b * MLP_NPARAM + p];
    grad[p] = a;
  }
  if (p == 0) {
    double l = 0.0;
    for (int b = 0; b < nblocks; ++b) l += loss_partial[b];
    *loss = l / (double)n;
  }
}

}  // namespace hydro

extern "C" int hydro_mlp_loss_grad_device(const float* weights, const float* x6, const float* target, long n,
                                          double* grad_out, double* loss_out, void* stream) {
  if (!weights || !x6 || !target || !grad_out || !loss_out)
    return berr("hydro_mlp_loss_grad_device: null pointer");
  if (n < 1 || n > hydro::NOALLOC_MAX_SAMPLES) {
    std::ostringstream m;
    m << "hydro_mlp_loss_grad_device: n = " << n << " outside [1, " << hydro::NOALLOC_MAX_SAMPLES
      << "] (the size of its static scratch)";
    return berr(m.str());
  }
  void* scratch = nullptr;
  int st = hydro::noalloc_scratch(&scratch);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  float* partial = (float*)scratch;
  double* loss_partial = (double*)((unsigned char*)scratch + hydro::NOALLOC_GRAD_BYTES);
  const int nblocks = (int)((n + MLP_SB - 1) / MLP_SB);
  mlp_grad_kernel<<<nblocks, 256, sizeof(MlpSmem), s>>>(weights, x6, target, nullptr, 0, n, (float)(1.0 / n),
                                                        partial, loss_partial);
  HCK(cudaGetLastError());
  hydro::noalloc_reduce_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(partial, loss_partial, nblocks, n,
                                                                       grad_out, loss_out);
  HCK(cudaGetLastError());
  return HYDRO_OK;
}
