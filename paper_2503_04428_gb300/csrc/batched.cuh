// batched.cuh -- thousands of independent 1D tubes advanced in one persistent launch.
//
// Each tube b is a uniform grid of n_b cells on [0,1] with transmissive ends
// and its own CFL time step dt_b = cfl / max_i (|u|+c) n_b (reading R4 in
// 1D).  The tubes are cut into work items of whole 28-cell segments; every
// warp of a persistent grid pulls items from an atomic counter and advances
// them on its own, with neighbour data exchanged by shuffles (no block-wide
// barrier on the step's path).  Per 28-cell segment, lane l of the warp:
//   - stages cell c0-2+l as primitives (Eq. 5);
//   - computes the limited slopes (Eq. 17) and Hancock increment (Eq. 18) of
//     cell c0-1+l and its two predicted face states;
//   - solves the exact Riemann problem (App. C.1) at face c0+l: identical
//     states give their own flux; elsewhere Toro's adaptive guess, replaced
//     by the MLP on faces where that rule picks the two-shock estimate for a
//     pressure jump above 4 (the warp evaluates the network together, one
//     such face at a time);
//     Newton to 1e-10 (FP64) and one polishing step; sample at x/t = 0;
//   - updates cell c0+l (Eq. 19) and reduces its signal speed.
// A segment whose whole window is one uniform state takes a short path that
// returns exactly what the full path returns there (U + 0).  The windows of
// BSPAN consecutive segments arrive together: one lane copies their aligned
// span of every variable into a slot of the warp's shared-memory ring with
// 1D bulk copies (cp.async.bulk, completion counted on the slot's mbarrier),
// several spans ahead of the one in use, so that enough bytes are in flight
// to cover HBM latency in few, large transfers.  Every variable's slab of
// the state starts on a 16-byte boundary for this (padded stride).  The
// network's weights arrive the same way, one bulk copy per CTA from a device
// copy kept in the kernel's shared-memory layout; only warps that meet a face
// using the network wait for them.
// One launch runs several steps.  Its queue holds every (step, item) entry,
// step by step, the items of a step in tube order; a tube's step waits only
// for the tube's own previous step (its time step is the tube's own CFL
// maximum), so there is no grid-wide barrier between steps: the warp that
// completes a tube's step commits it (time, speed slots) and releases the
// tube's next step.  With tube order the entries of a tube's next step come
// a whole step of other tubes' items later, so the release has normally
// happened when a warp takes them.
#pragma once
#include "common.cuh"

namespace hydro {

constexpr int BSEG = 28;   // cells per warp segment (32 lanes = 28 cells + 2 halo cells each side)
constexpr int BSPAN = 8;   // segments per ring slot
constexpr int BVSTR = 232; // elements per variable in a slot: the span's 228 cells widened to 16-byte bounds
constexpr int ST_TIMEOUT = -6;  // HYDRO_ERR_TIMEOUT: a bounded wait for a bulk copy expired

// Ring slots per warp (all but one in flight while one is in use): 3 in
// FP32 (4 measured no faster), 2 in FP64.
template <typename T>
__host__ __device__ constexpr int bdepth() {
  return sizeof(T) == 4 ? 3 : 2;
}
// Elements per 16 bytes: slabs, spans and copy sizes are multiples of this.
template <typename T>
__host__ __device__ constexpr int bquant() {
  return 16 / (int)sizeof(T);
}

// Dynamic shared memory of batched_kernel<T, NW>: one ring of bdepth<T>()
// slots (3 variables x BVSTR elements) per warp.
template <typename T, int NW>
constexpr size_t batched_smem_bytes() {
  return (size_t)NW * bdepth<T>() * 3 * BVSTR * sizeof(T);
}

// mbarrier and 1D bulk-copy primitives (PTX ISA: mbarrier, cp.async.bulk).
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* m) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(m)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(m))
               : "memory");
}
// Wait for phase `parity` of the mbarrier to complete, at most 2^20 polls
// (each poll may itself suspend the thread for a bounded time); false if it
// did not.
__device__ __forceinline__ bool mbar_wait(unsigned long long* m, unsigned parity) {
  const unsigned a = smem_addr(m);
  for (int i = 0; i < (1 << 20); ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// A tube's count of completed items, read with acquire semantics and
// raised with release semantics at GPU scope (PTX ISA memory consistency
// model): what a warp wrote before it counted its item is visible to a warp
// that has read the count.  The release follows a __syncwarp, so it covers
// the stores of every lane of the warp.
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void add_release(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
// Wait until count *p reaches n: 1 when it has, 0 when the launch failed
// meanwhile (status set), -1 when 2^22 polls (each with a short sleep,
// several seconds in all) did not see it.  (Out of line: a tube is normally
// ready when its item is taken; callers test the count first.)
static __device__ __noinline__ int tube_wait(const unsigned int* p, unsigned int n, const volatile Ctrl* vc) {
  for (int i = 0; i < (1 << 22); ++i) {
    if (ld_acquire(p) >= n) return 1;
    if (vc->status != 0) return 0;
    __nanosleep(256);
  }
  return -1;
}

// Exact-solver faces by where Newton started and in which precision it ran:
// Toro's guess, the network's guess (both in the form's precision), or the
// FP64 solve of an FP32 hard face (reading R12), whatever its guess.
enum { CAT_TORO = 0, CAT_MLP = 1, CAT_FP64 = 2, NCAT = 3 };

struct BatchCtrl {
  Ctrl c;
  unsigned long long next_entry;  // work-queue head of the running launch (entry = step x items + item)
  unsigned long long cat_faces[NCAT];  // faces that ran Newton, per category
  unsigned long long cat_iters[NCAT];  // their Newton iterations
};

struct MlpSmemW;

// One work item: cells beg .. end-1 of tube `tube` (nb cells, the first at
// element `base` of every variable's slab; the tube is cut into nit items),
// everything a warp needs before it issues the item's first copies, in one
// 32-byte record.
struct __align__(16) BatchItem {
  long long base;
  int nb;
  int beg;
  int end;
  int tube;
  int nit;
  int pad;
};
static_assert(sizeof(BatchItem) == 32, "one 32-byte record per item");

template <typename T>
struct BatchArgs {
  const T* A;
  T* B;
  T* Aw;
  long long stride;            // elements between the variables' slabs (a multiple of bquant<T>())
  const BatchItem* items;      // one step's work items, in hand-out order (tube order)
  int nitems;
  int nsteps;                  // steps of every tube in this launch
  int ntot;                    // tubes of the handle (the stride of smax)
  // Per tube b (s = the step count of a state):
  //   smax[(s % 3) * ntot + b]: bits of max_i (|u|+c)/h of the tube's state
  //     after s steps; step s collects its result's in slot (s + 1) % 3 and,
  //     in the tube's first item, clears slot (s + 2) % 3 for step s + 1;
  //   tcnt[b]: items of the tube completed in this launch (0 at its start);
  //   tstart[b]: 1 + the launch step whose dt the tube's first item added to
  //     t_tube (0 none; 0 at the launch's start);
  //   t_tube[b]: its time; t_prev[b]: its time before the last dt added.
  unsigned long long* smax;
  unsigned int* tcnt;
  int* tstart;
  double* t_tube;
  double* t_prev;
  double cfl;
  Gas<T> gas;
  int limiter;
  const MlpSmemW* mlp_w;        // packed weights (device) or null
  int mlp_on;
  double* harvest;             // capacity x 6 doubles or null
  unsigned long long* harvest_n;
  long long harvest_cap;
  unsigned long long harvest_thresh;
  unsigned long long harvest_seed;
  BatchCtrl* ctrl;
};

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  // SplitMix64 finaliser (Steele, Lea & Flood 2014)
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Network weights as the kernel holds them in shared memory; W2 is stored
// transposed (W2T[i][o]) so that the 32 lanes of a warp read consecutive
// words.  The host keeps a device copy in this layout (mlp_pack_kernel, run
// when the weights change), which every CTA loads with one bulk copy.
struct __align__(16) MlpSmemW {
  float w1[MLP_H * MLP_IN];
  float b1[MLP_H];
  float w2t[MLP_H * MLP_H];
  float b2[MLP_H];
  float w3[MLP_H];
  float b3;
  float pad[3];  // the size, a multiple of 16 bytes
};
static_assert(sizeof(MlpSmemW) % 16 == 0, "bulk-copied weights");

// The 4673 weights (flat layout of mlp.cuh) into the kernel's layout.
__global__ void mlp_pack_kernel(const float* __restrict__ w, MlpSmemW* __restrict__ out) {
  for (int p = threadIdx.x; p < MLP_H * MLP_IN; p += blockDim.x) out->w1[p] = w[MW1 + p];
  for (int p = threadIdx.x; p < MLP_H * MLP_H; p += blockDim.x) {
    const int o = p / MLP_H, i = p % MLP_H;
    out->w2t[i * MLP_H + o] = w[MW2 + p];
  }
  for (int p = threadIdx.x; p < MLP_H; p += blockDim.x) {
    out->b1[p] = w[MB1 + p];
    out->b2[p] = w[MB2 + p];
    out->w3[p] = w[MW3 + p];
  }
  if (threadIdx.x == 0) {
    out->b3 = w[MB3];
    out->pad[0] = out->pad[1] = out->pad[2] = 0.f;
  }
}

// The network's star-pressure guess for one face, evaluated by the whole
// warp: q = (rho_L, u_L, P_L, rho_R, u_R, P_R), the same on every lane; the
// features, the 6-64-64-1 network (lane l owns hidden units l and l+32) and
// the output y, returned with P_ref (the guess is P_ref exp(y)).  Out of line
// and compact (loops rolled, the features' logarithms and quotients and the
// activations' exponentials by the fast hardware approximations): few faces
// use it, and a longer body would crowd the instruction cache that every
// warp of the SM shares (measured: the cache's hit rate fell from 97 % to
// 87 % with the accurate forms inlined).  The guess only seeds Newton.
static __device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.0f + __expf(-z)); }
// (The face's six values come by value: an array passed to an out-of-line
// function lives in local memory, which cost the kernel spills in its hot
// loop; by value the loop needs none.)
static __device__ __noinline__ float2 mlp_guess_warp(const MlpSmemW& s, float g, float q0, float q1, float q2,
                                                     float q3, float q4, float q5, int lane) {
  const float q[6] = {q0, q1, q2, q3, q4, q5};
  float x[MLP_IN];
  const float rref = sqrtf(q[0] * q[3]), pref = sqrtf(q[2] * q[5]);
  const float icref = rsqrtf(g * __fdividef(pref, rref));
  x[0] = __logf(__fdividef(q[0], rref));
  x[1] = __logf(__fdividef(q[3], rref));
  x[2] = __logf(__fdividef(q[2], pref));
  x[3] = __logf(__fdividef(q[5], pref));
  x[4] = q[1] * icref;
  x[5] = q[4] * icref;
  float a = s.b1[lane], b = s.b1[lane + 32];
#pragma unroll 1
  for (int i = 0; i < MLP_IN; ++i) {
    a = fmaf(s.w1[lane * MLP_IN + i], x[i], a);
    b = fmaf(s.w1[(lane + 32) * MLP_IN + i], x[i], b);
  }
  const float ha = silu_fast(a), hb = silu_fast(b);
  float za = s.b2[lane], zb = s.b2[lane + 32];
#pragma unroll 1
  for (int i = 0; i < 32; ++i) {
    const float h0 = __shfl_sync(0xffffffffu, ha, i), h1 = __shfl_sync(0xffffffffu, hb, i);
    za = fmaf(s.w2t[i * MLP_H + lane], h0, za);
    za = fmaf(s.w2t[(i + 32) * MLP_H + lane], h1, za);
    zb = fmaf(s.w2t[i * MLP_H + lane + 32], h0, zb);
    zb = fmaf(s.w2t[(i + 32) * MLP_H + lane + 32], h1, zb);
  }
  float y = s.w3[lane] * silu_fast(za) + s.w3[lane + 32] * silu_fast(zb);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
  return make_float2(y + s.b3, pref);
}

// Value of lane (lane + off) of the 32-cell window (lanes beyond 31 are never used).
template <typename T>
__device__ __forceinline__ T win(T va, int off) {
  return __shfl_down_sync(0xffffffffu, va, off);
}

// Span k of item r: its 8 segments' windows (cells lo .. hi-1 of the tube,
// clamped to it: transmissive ends), widened to 16-byte bounds: elements
// g0 .. g0+len-1 of every variable's slab (len <= BVSTR).
template <typename T>
__device__ __forceinline__ void span_geom(const BatchItem& r, int k, long long& g0, int& len) {
  constexpr int Q = bquant<T>();
  const int lo = max(r.beg + k * BSPAN * BSEG - 2, 0);
  const int hi = min(r.beg + (k + 1) * BSPAN * BSEG + 2, r.nb);
  g0 = (r.base + lo) & ~(long long)(Q - 1);
  len = (int)(((r.base + hi + Q - 1) & ~(long long)(Q - 1)) - g0);
}

// Span k of item r into a ring slot (3 variables, BVSTR elements apart), one
// bulk copy per variable completing on the slot's mbarrier (issued by one
// lane).
template <typename T>
__device__ __forceinline__ void issue_span(T* slotp, unsigned long long* bar, const T* Uin, long long stride,
                                           const BatchItem& r, int k) {
  long long g0;
  int len;
  span_geom<T>(r, k, g0, len);
  const unsigned bytes = (unsigned)len * (unsigned)sizeof(T);
  mbar_expect_tx(bar, 3u * bytes);
#pragma unroll
  for (int v = 0; v < 3; ++v) bulk_copy_g2s(slotp + v * BVSTR, Uin + v * stride + g0, bytes, bar);
}

// A state that repeats over a whole window (the uniform shortcut): its |u|
// + c and its validity (0 or a status).  Out of line: it runs once per new
// uniform state, and the kernel's hot code stays shorter.  (Results come by
// value: a local whose address an out-of-line function takes lives in local
// memory.)
template <typename T>
struct SpeedSt {
  T s;
  int st;
};
template <typename T>
static __device__ __noinline__ SpeedSt<T> uniform_speed(T r0, T r1, T r2, Gas<T> gas) {
  T u[3] = {r0 + T(0), r1 + T(0), r2 + T(0)}, w[3];
  const bool finite = isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
  to_prim<T, 1, 0>(u, w, gas);
  SpeedSt<T> r;
  r.st = !finite ? ST_NONFINITE : (!(w[0] > T(0)) || !(w[2] > T(0))) ? ST_NEG : 0;
  r.s = fabs(w[1]) + dsqrt(qdiv(gas.g * w[2], w[0]));
  return r;
}

// Record a gated face's states (network training data) with probability
// thresh / 2^64, counter-based per face id and step.  Out of line: it runs
// only while harvesting.
template <typename T, typename A>
static __device__ __noinline__ void harvest_face(const A& a, unsigned long long id, long long step, T l0, T l1,
                                                 T l2, T r0, T r1, T r2) {
  const T WL[3] = {l0, l1, l2}, WR[3] = {r0, r1, r2};
  const unsigned long long hsh =
      mix64(a.harvest_seed + 0x9E3779B97F4A7C15ull * (id + 1) + ((unsigned long long)step << 40));
  if (hsh < a.harvest_thresh) {
    const unsigned long long slot = atomicAdd(a.harvest_n, 1ull);
    if ((long long)slot < a.harvest_cap) {
      for (int v = 0; v < 3; ++v) {
        a.harvest[slot * 6 + v] = (double)WL[v];
        a.harvest[slot * 6 + 3 + v] = (double)WR[v];
      }
    }
  }
}

// Two register budgets for the autotuner: 8-warp CTAs with 2 resident per SM
// (128 registers) and 4-warp CTAs with 5 per SM (about 100).
template <typename T, int NW>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 2 : 5)
    batched_kernel(const BatchArgs<T> a) {
  __shared__ MlpSmemW sw;
  __shared__ unsigned long long wbar;  // completes when sw has landed
  extern __shared__ __align__(16) unsigned char ring_raw[];
  const volatile Ctrl* vc = &a.ctrl->c;
  // the buffer of the state at the launch's start and the steps every tube
  // had completed then (in shared memory: read where needed); a launch
  // behind a failed one does nothing (one read for the whole CTA)
  __shared__ long long s_step0;
  __shared__ int s_cur0, s_fail;
  if (threadIdx.x == 0) {
    s_fail = vc->status;
    s_step0 = vc->step;
    s_cur0 = vc->cur;
  }
  __syncthreads();
  if (s_fail != 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int BD = bdepth<T>(), Q = bquant<T>();
  T* ring = reinterpret_cast<T*>(ring_raw) + warp * (BD * 3 * BVSTR);
  __shared__ unsigned long long bar[NW][BD];  // one mbarrier per ring slot
  if (lane < BD) mbar_init(&bar[warp][lane]);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // the inits, visible to the copies
  __syncwarp();
  const Gas<T>& gas = a.gas;
  // the network's weights arrive by one bulk copy; only warps that meet a
  // face using the network wait for them
  if (a.mlp_on) {
    if (threadIdx.x == 0) {
      mbar_init(&wbar);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_expect_tx(&wbar, (unsigned)sizeof(MlpSmemW));
      bulk_copy_g2s(&sw, a.mlp_w, (unsigned)sizeof(MlpSmemW), &wbar);
    }
  }
  __syncthreads();  // the launch's start values (and the weights' barrier), visible to every warp
  bool w_ready = false;  // this warp has seen the weights land
  unsigned long long n_iters = 0, n_mlp = 0, n_fb = 0;
  unsigned cat_f[NCAT] = {0u, 0u, 0u}, cat_i[NCAT] = {0u, 0u, 0u};  // per-lane counts of this launch
  int err = 0;
  // the last uniform window's state and its |u| + c (warp-uniform values)
  bool have_u = false;
  T ur[3] = {T(0), T(0), T(0)}, u_spd = T(0);
  // spans issued into / taken out of this warp's ring so far (warp-uniform);
  // slot q % BD completes its phase (q / BD) & 1 for the q-th span
  unsigned q_issue = 0, q_use = 0;
  bool dead = false;  // a bounded wait expired: stop, drain, report

  const unsigned long long nent = (unsigned long long)a.nitems * (unsigned long long)a.nsteps;
  for (;;) {
    // Take the next entry; wait (bounded) until its tube's previous step is
    // complete (a step of the launch after the first); a failed launch stops
    // here.  Then the step's dt; the tube's first item also advances the
    // tube's time by dt and clears the speed slot that the next step
    // collects into (every item of the previous step has read it).
    int go = 1;
    BatchItem itm;
    int lstep = 0;
    double dtd = 0.0;
    if (lane == 0) {
      const unsigned long long e = atomicAdd(&a.ctrl->next_entry, 1ull);
      if (e >= nent) {
        go = 0;  // the queue is empty
      } else if (vc->status != 0) {
        go = 2;
      } else {
        lstep = (int)(e / (unsigned long long)a.nitems);
        itm = a.items[(int)(e - (unsigned long long)lstep * (unsigned long long)a.nitems)];
        const unsigned int need = (unsigned int)lstep * (unsigned int)itm.nit;
        if (lstep > 0 && ld_acquire(&a.tcnt[itm.tube]) < need) {
          const int r = tube_wait(&a.tcnt[itm.tube], need, vc);
          if (r != 1) go = r < 0 ? -1 : 2;
        }
        if (go == 1) {
          // the writes released with the count, visible to the bulk copies
          asm volatile("fence.proxy.async.global;\n" ::: "memory");
          const long long sm = (s_step0 + lstep) % 3;
          dtd = a.cfl / __longlong_as_double((long long)__ldcg(&a.smax[sm * a.ntot + itm.tube]));
          if (itm.beg == 0) {
            const double t = __ldcg(&a.t_tube[itm.tube]);
            a.t_prev[itm.tube] = t;
            a.t_tube[itm.tube] = t + dtd;
            a.tstart[itm.tube] = lstep + 1;
            a.smax[((sm + 2) % 3) * a.ntot + itm.tube] = 0ull;
          }
        }
      }
    }
    go = __shfl_sync(0xffffffffu, go, 0);
    if (go != 1) {
      if (go < 0 && lane == 0 && atomicCAS(&a.ctrl->c.status, 0, ST_TIMEOUT) == 0)
        a.ctrl->c.err_step = s_step0 + lstep;
      break;
    }
    // the item's record, from lane 0 to the warp
    itm.base = __shfl_sync(0xffffffffu, itm.base, 0);
    itm.nb = __shfl_sync(0xffffffffu, itm.nb, 0);
    itm.beg = __shfl_sync(0xffffffffu, itm.beg, 0);
    itm.end = __shfl_sync(0xffffffffu, itm.end, 0);
    itm.tube = __shfl_sync(0xffffffffu, itm.tube, 0);
    lstep = __shfl_sync(0xffffffffu, lstep, 0);
    dtd = __shfl_sync(0xffffffffu, dtd, 0);
    const long long step = s_step0 + lstep;
    const int b = itm.tube;
    const bool odd = ((s_cur0 ^ lstep) & 1) != 0;
    const T* Uin = odd ? a.B : a.A;
    T* Uout = odd ? a.Aw : a.B;
    const int s_beg = itm.beg, s_end = itm.end, nb = itm.nb;
    const long long base = itm.base;
    const T fn = (T)nb;          // 1/h
    const T hw = T(0.5) / fn;    // half width
    T smax = T(0);
    T* const out = Uout + base;  // the tube's cell 0 in the output

    // The conserved windows (cells c0-2+lane, clamped to the tube) of
    // segments BSPAN*k .. BSPAN*k+BSPAN-1 arrive in ring slot q_use % BD as
    // span k (span_geom), BD-1 spans ahead of the one in use.
    const int nseg = (s_end - s_beg + BSEG - 1) / BSEG;
    const int nspan = (nseg + BSPAN - 1) / BSPAN;
    for (int k = 0; k < BD - 1 && k < nspan; ++k) {
      if (lane == 0) issue_span<T>(ring + (q_issue % BD) * (3 * BVSTR), &bar[warp][q_issue % BD], Uin, a.stride,
                                   itm, k);
      ++q_issue;
    }
    const T dtdx = (T)dtd * fn;
    for (int k = 0; k < nspan; ++k) {
      __syncwarp();  // every lane is done with the slot refilled next (read one span ago)
      if (k + BD - 1 < nspan) {
        if (lane == 0) issue_span<T>(ring + (q_issue % BD) * (3 * BVSTR), &bar[warp][q_issue % BD], Uin,
                                     a.stride, itm, k + BD - 1);
        ++q_issue;
      }
      const int sl = (int)(q_use % BD);
      const bool landed = mbar_wait(&bar[warp][sl], (q_use / BD) & 1u);
      if (__any_sync(0xffffffffu, !landed)) {
        // q_use still names the span whose wait expired: the drain below
        // waits for it again, with the later spans already issued
        dead = true;
        err = ST_TIMEOUT;
        break;
      }
      ++q_use;
      long long g0;
      int len;
      span_geom<T>(itm, k, g0, len);
      const T* slot = ring + sl * (3 * BVSTR);
      const int ib = (int)(base - g0);  // slot index of the tube's cell 0
      // A span whose whole window (every cell any of its segments reads) is
      // one state: each of its cells gets U + 0, what the segment paths
      // below give there.  Tested against the span's first cell, with a few
      // strided shared-memory reads per lane and one vote; the state's
      // validity and |u| + c are cached like a uniform segment's.
      {
        const int i0 = ib + max(s_beg + k * BSPAN * BSEG - 2, 0);
        const int i1 = ib + min(s_beg + (k + 1) * BSPAN * BSEG + 2, nb);
        const T r0 = slot[i0], r1 = slot[BVSTR + i0], r2 = slot[2 * BVSTR + i0];
        bool eq = true;
        for (int i = i0 + lane; i < i1; i += 32)
          eq = eq & (slot[i] == r0) & (slot[BVSTR + i] == r1) & (slot[2 * BVSTR + i] == r2);
        if (__all_sync(0xffffffffu, eq)) {
          if (!(have_u & (r0 == ur[0]) & (r1 == ur[1]) & (r2 == ur[2]))) {
            have_u = true;
            ur[0] = r0;
            ur[1] = r1;
            ur[2] = r2;
            const SpeedSt<T> us = uniform_speed<T>(r0, r1, r2, gas);
            u_spd = us.s;
            if (err == 0) err = us.st;
          }
          smax = fmax(smax, u_spd * fn);
          const int a0 = s_beg + k * BSPAN * BSEG, a1 = min(a0 + BSPAN * BSEG, s_end);
          const T o0 = ur[0] + T(0), o1 = ur[1] + T(0), o2 = ur[2] + T(0);
          for (int c = a0 + lane; c < a1; c += 32) {
            out[c] = o0;
            out[a.stride + c] = o1;
            out[2 * a.stride + c] = o2;
          }
          continue;
        }
      }
#pragma unroll 1
      for (int j = 0; j < BSPAN; ++j) {
        const int sg = k * BSPAN + j;
        if (sg >= nseg) break;
        const int c0 = s_beg + sg * BSEG;
        T Ua[3];
        {
          const int idx = ib + min(max(c0 - 2 + lane, 0), nb - 1);
#pragma unroll
          for (int v = 0; v < 3; ++v) Ua[v] = slot[v * BVSTR + idx];
        }
        const int ncell = min(BSEG, s_end - c0);  // cells updated in this segment
        // A window holding one state everywhere (clamped tube ends included)
        // has zero slopes, a +0 Hancock increment, identical face states and
        // equal fluxes, so the full path below returns U + 0 for every cell:
        // produce exactly that without the face work.  First test against
        // the last uniform window's state (the common case along the
        // undisturbed stretch of a tube: no shuffles), then against lane 0.
        // (every vote and shuffle runs on every lane: a collective inside a
        // short-circuit condition would leave lanes out of it)
        bool uniform = __all_sync(0xffffffffu, have_u & (Ua[0] == ur[0]) & (Ua[1] == ur[1]) & (Ua[2] == ur[2]));
        if (!uniform) {
          const T r0 = __shfl_sync(0xffffffffu, Ua[0], 0);
          const T r1 = __shfl_sync(0xffffffffu, Ua[1], 0);
          const T r2 = __shfl_sync(0xffffffffu, Ua[2], 0);
          uniform = __all_sync(0xffffffffu, (Ua[0] == r0) & (Ua[1] == r1) & (Ua[2] == r2));
          if (uniform) {
            // a new uniform state: its validity and |u| + c, kept for the
            // windows that repeat it
            have_u = true;
            ur[0] = r0;
            ur[1] = r1;
            ur[2] = r2;
            const SpeedSt<T> us = uniform_speed<T>(r0, r1, r2, gas);
            u_spd = us.s;
            if (err == 0) err = us.st;
          }
        }
        if (uniform) {
          // (equal values compare equal but for the sign of zero, which
          // U + 0 erases: the cached state's U + 0 is the window's)
          smax = fmax(smax, u_spd * fn);
          if (lane < ncell) {
            T* o = out + c0 + lane;
            o[0] = ur[0] + T(0);
            o[a.stride] = ur[1] + T(0);
            o[2 * a.stride] = ur[2] + T(0);
          }
          continue;
        }
        // a1 + a2: primitives of the window (transmissive ends by clamping)
        T Wa[3];
        to_prim<T, 1, 0>(Ua, Wa, gas);
        // a3 + a4: cell c0-1+lane -- slopes, Hancock increment, predicted face states
        T Wc[3], Wlo[3], Whi[3];
        {
          T Wp[3], fl[3], fh[3];
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            Wc[v] = win(Wa[v], 1);
            Wp[v] = win(Wa[v], 2);
            const T sig = limit<T>(a.limiter, (Wc[v] - Wa[v]) * fn, (Wp[v] - Wc[v]) * fn);
            Wlo[v] = Wc[v] - hw * sig;
            Whi[v] = Wc[v] + hw * sig;
          }
          phys_flux<T, 1, 0, 0>(Wlo, fl, gas);
          phys_flux<T, 1, 0, 0>(Whi, fh, gas);
          T ul[3], uh[3];
          to_cons<T, 1, 0>(Wlo, ul, gas);
          to_cons<T, 1, 0>(Whi, uh, gas);
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            const T du = T(0.5) * dtdx * (fl[v] - fh[v]);
            ul[v] += du;
            uh[v] += du;
          }
          to_prim<T, 1, 0>(ul, Wlo, gas);
          to_prim<T, 1, 0>(uh, Whi, gas);
          // a non-physical prediction falls back to the cell average
          const bool own = lane >= 1 && lane <= ncell;  // cells of this segment
          if (!(Wlo[0] > T(0)) || !(Wlo[2] > T(0))) {
#pragma unroll
            for (int v = 0; v < 3; ++v) Wlo[v] = Wc[v];
            if (own) ++n_fb;
          }
          if (!(Whi[0] > T(0)) || !(Whi[2] > T(0))) {
#pragma unroll
            for (int v = 0; v < 3; ++v) Whi[v] = Wc[v];
            if (own) ++n_fb;
          }
        }
        // a5: face c0+lane between cell c0-1+lane (its high state, this lane)
        // and cell c0+lane (its low state, next lane)
        T WL[3], WR[3], F[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          WL[v] = Whi[v];
          WR[v] = __shfl_down_sync(0xffffffffu, Wlo[v], 1);
        }
        const bool face = lane <= ncell;
        const bool owned = face && (lane < ncell || c0 + lane == nb);
        const bool same = WL[0] == WR[0] && WL[1] == WR[1] && WL[2] == WR[2];
        T pg = T(0);
        int kind = 0;
        bool by_mlp = false;  // pg came from the network
        T cL = T(0), cR = T(0);
        if (face && !same) {
          cL = dsqrt(qdiv(gas.g * WL[2], WL[0]));
          cR = dsqrt(qdiv(gas.g * WR[2], WR[0]));
          pg = toro_guess<T>(WL[0], WL[1], WL[2], cL, WR[0], WR[1], WR[2], cR, gas, kind);
          if (!mlp_gate<T>(kind, WL[2], WR[2])) kind = -kind;  // negative: network not used
          if (kind == 2 && a.harvest)
            harvest_face<T, BatchArgs<T>>(a, (unsigned long long)(base + b + c0 + lane), step, WL[0], WL[1], WL[2],
                                          WR[0], WR[1], WR[2]);
        }
        // learned guess on two-shock faces, evaluated by the whole warp
        if (a.mlp_on) {
          unsigned todo = __ballot_sync(0xffffffffu, face && !same && kind == 2);
          if (todo && !w_ready) {
            w_ready = __all_sync(0xffffffffu, mbar_wait(&wbar, 0u));
            if (!w_ready) {
              err = ST_TIMEOUT;  // (these faces keep Toro's guess)
              todo = 0u;
            }
          }
          while (todo) {
            const int g = __ffs(todo) - 1;
            todo &= todo - 1;
            float q[6];
#pragma unroll
            for (int v = 0; v < 3; ++v) {
              q[v] = (float)__shfl_sync(0xffffffffu, WL[v], g);
              q[3 + v] = (float)__shfl_sync(0xffffffffu, WR[v], g);
            }
            const float2 yp = mlp_guess_warp(sw, (float)gas.g, q[0], q[1], q[2], q[3], q[4], q[5], lane);
            if (lane == g) {
              // (the guess only seeds Newton: FP32 exp in the FP32 form)
              if constexpr (sizeof(T) == 4) pg = yp.y * __expf(yp.x);
              else pg = (T)((double)yp.y * exp((double)yp.x));
              by_mlp = true;
              if (owned) ++n_mlp;
            }
          }
        }
        if (face) {
          if (same) {
            phys_flux<T, 1, 0, 0>(WL, F, gas);
          } else {
            // from the guess and sound speeds chosen above (Newton starts
            // from the same value the general entry would use)
            int its = 0;
            const int st = riemann_exact_from<T>(WL, WR, cL, cR, pg, F, gas, its);
            if (owned) {
              n_iters += its;
              int cat = by_mlp ? CAT_MLP : CAT_TORO;
              if constexpr (sizeof(T) == 4) {
                if (hard_face<T>(WL[2], WR[2], WR[1] - WL[1], gas.two_gm1 * (cL + cR))) cat = CAT_FP64;
              }
              cat_f[cat] += 1u;
              cat_i[cat] += (unsigned)its;
            }
            if (st != ST_OK && err == 0) err = st;
          }
        }
        // a6: update cell c0+lane with faces c0+lane (this lane) and c0+lane+1 (next)
        T Fh[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) Fh[v] = __shfl_down_sync(0xffffffffu, F[v], 1);
        T Uo[3];  // conserved state of cell c0+lane, from the window (lane+2)
#pragma unroll
        for (int v = 0; v < 3; ++v) Uo[v] = win(Ua[v], 2);
        if (lane < ncell) {
          const long long c = base + c0 + lane;
          T u[3], w[3];
          bool finite = true;
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            u[v] = Uo[v] + dtdx * (F[v] - Fh[v]);
            finite = finite && isfinite(u[v]);
          }
          to_prim<T, 1, 0>(u, w, gas);
          if (!finite) err = err ? err : ST_NONFINITE;
          else if (!(w[0] > T(0)) || !(w[2] > T(0))) err = err ? err : ST_NEG;
          smax = fmax(smax, (fabs(w[1]) + dsqrt(qdiv(gas.g * w[2], w[0]))) * fn);
#pragma unroll
          for (int v = 0; v < 3; ++v) Uout[v * a.stride + c] = u[v];
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    // A failure stops the launch before the tube completes the step: its
    // state stays that of the previous step.
    int ferr = err;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int e2 = __shfl_xor_sync(0xffffffffu, ferr, o);
      ferr = ferr ? ferr : e2;
    }
    if (dead || ferr) {
      if (lane == 0 && atomicCAS(&a.ctrl->c.status, 0, ferr ? ferr : ST_TIMEOUT) == 0) a.ctrl->c.err_step = step;
      break;
    }
    // The item is complete: its speed maximum, then its count (a release:
    // every lane's stores of the item come first).
    __syncwarp();
    if (lane == 0) {
      atomicMax(&a.smax[((step + 1) % 3) * a.ntot + b], dbits((double)smax));
      add_release(&a.tcnt[b], 1u);
    }
  }
  // after an expired wait, let the copies still in flight land (bounded)
  // before the CTA's shared memory is released: spans q_use .. q_issue-1,
  // the one whose wait expired first (on a normal exit q_use == q_issue)
  while (q_use < q_issue) {
    mbar_wait(&bar[warp][q_use % BD], (q_use / BD) & 1u);
    ++q_use;
  }

  // block totals of the counters and the error, then the last-CTA commit
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_iters += __shfl_xor_sync(0xffffffffu, n_iters, o);
    n_mlp += __shfl_xor_sync(0xffffffffu, n_mlp, o);
    n_fb += __shfl_xor_sync(0xffffffffu, n_fb, o);
#pragma unroll
    for (int c = 0; c < NCAT; ++c) {
      cat_f[c] += __shfl_xor_sync(0xffffffffu, cat_f[c], o);
      cat_i[c] += __shfl_xor_sync(0xffffffffu, cat_i[c], o);
    }
    const int e2 = __shfl_xor_sync(0xffffffffu, err, o);
    err = err ? err : e2;
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < NCAT; ++c) {
      if (cat_f[c]) atomicAdd(&a.ctrl->cat_faces[c], (unsigned long long)cat_f[c]);
      if (cat_i[c]) atomicAdd(&a.ctrl->cat_iters[c], (unsigned long long)cat_i[c]);
    }
    if (n_iters) atomicAdd(&a.ctrl->c.iters, n_iters);
    if (n_mlp) atomicAdd(&a.ctrl->c.mlp, n_mlp);
    if (n_fb) atomicAdd(&a.ctrl->c.fallbacks, n_fb);
    if (err && atomicCAS(&a.ctrl->c.status, 0, err) == 0) a.ctrl->c.err_step = -1;
  }
  // the weights' copy has landed before the CTA ends (bounded)
  if (a.mlp_on && threadIdx.x == 0) mbar_wait(&wbar, 0u);
  __syncthreads();
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&a.ctrl->c.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  // the last CTA: every tube has completed the launch's steps (or the launch
  // failed, and the host settles the tubes)
  __threadfence();
  volatile BatchCtrl* vb = a.ctrl;
  if (vb->c.status == 0) {
    vb->c.step = s_step0 + a.nsteps;
    vb->c.cur = s_cur0 ^ (a.nsteps & 1);
  }
  vb->c.done = 0;
  vb->next_entry = 0ull;
  __threadfence();
}

// max_i (|u|+c)/h over cells lo .. lo+n-1 of slab-strided state U (this
// thread's share, strided by blockDim.x), reduced over the CTA (FP64);
// thread 0 receives the maximum and the first invalid cell's status.
template <typename T>
__device__ void tube_speed(const T* U, long long stride, long long lo, int n, const Gas<T>& gas, double& m,
                           int& e) {
  double smax = 0.0;
  int err = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T u[3], w[3];
    bool finite = true;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      u[v] = U[v * stride + lo + i];
      finite = finite && isfinite(u[v]);
    }
    if (!finite) { err = ST_NONFINITE; continue; }
    to_prim<T, 1, 0>(u, w, gas);
    if (!(w[0] > T(0)) || !(w[2] > T(0))) { err = err ? err : ST_NEG; continue; }
    smax = fmax(smax, (double)((fabs(w[1]) + dsqrt(gas.g * w[2] / w[0])) * (T)n));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    const int e2 = __shfl_xor_sync(0xffffffffu, err, o);
    err = err ? err : e2;
  }
  __shared__ double red_s[32];
  __shared__ int red_e[32];
  if ((threadIdx.x & 31) == 0) {
    red_s[threadIdx.x >> 5] = smax;
    red_e[threadIdx.x >> 5] = err;
  }
  __syncthreads();
  m = 0.0;
  e = 0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      m = fmax(m, red_s[k]);
      e = e ? e : red_e[k];
    }
  }
}

// A new state's per-tube bookkeeping, one CTA per tube (tubes tube0 ..
// tube0+ntubes-1): with s = ctrl->step, speed slot s % 3 gets max_i
// (|u|+c)/h (FP64 bits) and the other two slots 0; the tube has no item of
// a launch completed and its time is 0.  An invalid cell sets *status.  In
// one pass over the tube, so a host-resident run needs no copy or memset
// between its input copy and its steps.  (blockDim.x: a multiple of 32, at
// most 1024.)
template <typename T>
__global__ void batch_init_kernel(const T* U, long long stride, const long long* off, int tube0, int ntubes,
                                  Gas<T> gas, const Ctrl* ctrl, int ntot, unsigned long long* smax,
                                  unsigned int* tcnt, int* tstart, double* t_tube, double* t_prev, int* status) {
  if ((int)blockIdx.x >= ntubes) return;
  const int b = tube0 + blockIdx.x;
  const long long base = off[b];
  double m;
  int e;
  tube_speed<T>(U, stride, base, (int)(off[b + 1] - base), gas, m, e);
  if (threadIdx.x == 0) {
    const long long s = ctrl->step;
#pragma unroll
    for (int k = 0; k < 3; ++k) smax[((s + k) % 3) * ntot + b] = k == 0 ? dbits(m) : 0ull;
    tcnt[b] = 0u;
    tstart[b] = 0;
    t_tube[b] = 0.0;
    t_prev[b] = 0.0;
    if (e) atomicCAS(status, 0, e);
  }
}

// After a failed launch that started at step count s0 with the state in
// buffer cur0 (items of item_len cells): tube b completed k = tcnt[b] / nit
// of its steps, so its last good state is in buffer cur0 ^ (k & 1).  Move it
// to buffer cur0, where every tube's state then is; take back the dt of a
// step that started but did not complete (tstart); restart the speed slots
// at step count s0 with the tube's speed recomputed.
template <typename T>
__global__ void batch_settle_kernel(T* A, T* B, long long stride, const long long* off, int item_len, Gas<T> gas,
                                    long long s0, int cur0, int ntot, unsigned long long* smax, unsigned int* tcnt,
                                    int* tstart, double* t_tube, const double* t_prev) {
  const int b = blockIdx.x;
  const long long base = off[b];
  const int nb = (int)(off[b + 1] - base);
  T* dst = cur0 ? B : A;
  const T* src = cur0 ? A : B;
  const int nit = (nb + item_len - 1) / item_len;
  const int k = (int)(tcnt[b] / (unsigned int)nit);
  if (k & 1) {
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
#pragma unroll
      for (int v = 0; v < 3; ++v) dst[v * stride + base + i] = src[v * stride + base + i];
  }
  double m;
  int e;
  tube_speed<T>(dst, stride, base, nb, gas, m, e);  // (each thread reads the cells it copied)
  if (threadIdx.x == 0) {
    if (tstart[b] - 1 >= k) t_tube[b] = t_prev[b];
#pragma unroll
    for (int j = 0; j < 3; ++j) smax[((s0 + j) % 3) * ntot + b] = j == 0 ? dbits(m) : 0ull;
    tcnt[b] = 0u;
    tstart[b] = 0;
  }
}

// Interior faces of the tubes whose two cells hold different states (those
// that need the Riemann solver), counted into *count; one CTA per tube.
// (blockDim.x: a multiple of 32, at most 1024.)
template <typename T>
__global__ void batch_rough_kernel(const T* U, long long stride, const long long* off, unsigned long long* count) {
  const int b = blockIdx.x;
  const long long base = off[b];
  const int nb = (int)(off[b + 1] - base);
  unsigned int c = 0;
  for (int i = 1 + threadIdx.x; i < nb; i += blockDim.x) {
    bool same = true;
#pragma unroll
    for (int v = 0; v < 3; ++v) same = same && U[v * stride + base + i] == U[v * stride + base + i - 1];
    c += same ? 0u : 1u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

// Exact star states of independent faces (one thread per face).
template <typename T>
__global__ void exact_list_kernel(const double* WL, const double* WR, long long n, Gas<T> gas,
                                  const float* mlp_w, double* pstar, double* ustar, int* iters) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T rL = (T)WL[3 * i], uL = (T)WL[3 * i + 1], pL = (T)WL[3 * i + 2];
  const T rR = (T)WR[3 * i], uR = (T)WR[3 * i + 1], pR = (T)WR[3 * i + 2];
  T guess = T(0);
  if (mlp_w) {
    const T cL = dsqrt(gas.g * pL / rL), cR = dsqrt(gas.g * pR / rR);
    int kind;
    toro_guess<T>(rL, uL, pL, cL, rR, uR, pR, cR, gas, kind);
    if (mlp_gate<T>(kind, pL, pR)) {
      float x[6], pref;
      mlp_features((float)gas.g, (float)rL, (float)uL, (float)pL, (float)rR, (float)uR, (float)pR, x, pref);
      guess = (T)((double)pref * exp((double)mlp_forward(mlp_w, x)));
    }
  }
  T ps = T(0), us = T(0);
  int its = 0, kind = 0;
  const int st = exact_star<T>(rL, uL, pL, rR, uR, pR, gas, guess, ps, us, its, kind);
  pstar[i] = st == ST_OK ? (double)ps : -1.0;
  ustar[i] = (double)us;
  iters[i] = st == ST_OK ? its : -st;
}

// The exact solution of face face_of[k] at x/t = xi[k], in FP64, from the
// star states of exact_list_kernel: W_out[3k..3k+2] = (rho, u, P).
__global__ void exact_sample_kernel(const double* WL, const double* WR, const double* pstar,
                                    const double* ustar, const long long* face_of, const double* xi,
                                    long long npts, Gas<double> gas, double* W_out) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= npts) return;
  const long long f = face_of[k];
  const double rL = WL[3 * f], uL = WL[3 * f + 1], pL = WL[3 * f + 2];
  const double rR = WR[3 * f], uR = WR[3 * f + 1], pR = WR[3 * f + 2];
  const double cL = sqrt(gas.g * pL / rL), cR = sqrt(gas.g * pR / rR);
  double rho, u, p;
  sample_xi<double>(xi[k], rL, uL, pL, cL, rR, uR, pR, cR, pstar[f], ustar[f], gas, rho, u, p);
  W_out[3 * k] = rho;
  W_out[3 * k + 1] = u;
  W_out[3 * k + 2] = p;
}

}  // namespace hydro
