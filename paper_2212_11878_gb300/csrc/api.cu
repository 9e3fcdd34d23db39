// api.cu -- host runtime behind include/mpcd.h: handle lifetime, parameter checks, device
// buffers, the per-step launch sequence (replayed from a captured CUDA graph), per-kernel
// event timing and error reporting.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "mpcd.h"
#include "cellmath.cuh"
#include "device_common.cuh"
#include "mpcd_internal.h"

using namespace mpcd;

namespace {

enum KernelSlot {
  kSlotZero = 0,
  kSlotStreamBin,
  kSlotScan,
  kSlotScatter,
  kSlotCollide,
  kSlotRotate,
  kSlotEndStep,
  kSlotRotateStream,
  kSlotStep,
  kNumSlots
};
const char* kSlotNames[kNumSlots] = {"zero_counts", "stream_bin", "scan",     "scatter",       "collide",
                                     "rotate",      "end_step",   "rotate_stream", "step"};
// kernels launched per invocation of each slot (the rotation slots only for the dense pair;
// "step" is the mixed form's one-launch step)
const int kSlotLaunchesBase[kNumSlots] = {1, 1, 3, 1, 1, 0, 1, 0, 1};

// The launch sequence of one step.  Full: every kernel of a step (mixed form, and FP64 boxes
// whose collision is one per-cell kernel).  The FP64 dense pair splits its steps so that the
// rotation of step t runs fused with the streaming of step t + 1: an mpcd_step(n) call is a
// Head (step 1 up to its frames), n - 1 Bodies (the rotation of the previous step fused with
// the streaming of this one, then this step up to its frames) and a Tail (the last rotation),
// so that no call leaves a step half done.  With the tuning's fuse = 0 every step of the
// dense pair is a Step: Full, then its own rotation.
enum Piece { kPieceFull = 0, kPieceBody = 1, kPieceTail = 2, kPieceStep = 3 };  // Step: Full + Tail

// Message of the last failure without a handle (create, the allocation-free step), one slot
// per calling thread.
thread_local std::string g_create_err;

struct PendingTiming {
  int slot;
  cudaEvent_t a, b;
};

}  // namespace

struct mpcd_s {
  int device = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  int precision = MPCD_FP64;
  int nbox = 1;
  Geom geom{};
  int64_t n = 0, ncell = 0;
  Fp64Bufs f64{};
  double* host_stage = nullptr;  // 6 N doubles for the host get/set_state copies, made on first use
  cudaStream_t copy_stream = nullptr;  // FP64 host get_state: chunk copies beside the gathers
  std::vector<cudaEvent_t> chunk_events;
  double* mass_buf[3] = {};  // FP64 particle masses: storage order (two buffer sets), id order
  Fp64Mass f64m{};           // points at mass_buf[0..1] while masses are set
  float* mix_mass_buf[2] = {};  // mixed form: FP32 masses in the storage order of each record buffer
  MixMass mixm{};               // points at mix_mass_buf while masses are set
  bool masses = false;
  Scratch scr{};
  MixBufs mix{};
  MixScratch mscr{};
  bool mixed_keys_valid = false;  // keys and counts of the next step exist (mixed form)
  // mixed form: per-box tables (host copies and device arrays)
  std::vector<Geom> boxes;
  std::vector<int64_t> pbase;
  Geom* d_boxes = nullptr;
  BoxShift* d_shifts = nullptr;
  MixGroup* d_groups = nullptr;       // rewritten every step by k_group_bounds
  MixGroupSpec* d_gspec = nullptr;    // fixed part of the group table
  int64_t* d_pbase = nullptr;
  int64_t groups_cap = 0;
  MixBatch mb{};
  mpcd_tuning tune{};
  Ctl* ctl = nullptr;
  unsigned long long* d_bad = nullptr;  // first invalid particle found by the state check
  unsigned* d_bar = nullptr;            // grid-barrier counters of the one-launch mixed step
  int stall_test = 0;                   // test hook: the next one-launch step's barriers run out
  Ctl ctl_host{};  // host copy used to (re)initialise the device control block
  int red_blocks = 0;
  std::vector<void*> allocations;

  // host mirror of the device step control
  int64_t t = 0;
  int cur = 0;
  bool last_resorted = false;
  bool any_step = false;
  bool perm_sorted = false;  // perm of the last step is in storage order inside each cell

  bool record_moments = false;
  bool moments_valid = false;

  cudaGraphExec_t graph = nullptr;       // FP64: one step (the dense pair: up to its frames)
  cudaGraphExec_t graph_body = nullptr;  // FP64 dense pair: the fused body of a step
  cudaGraphExec_t graph_step = nullptr;  // FP64 dense pair, unfused: a step with its rotation
  cudaGraphExec_t graph_par[2] = {};     // mixed: one step starting from buffer set 0 / 1
  bool graph_moments = false;

  bool timing = false;
  std::vector<PendingTiming> pending;
  std::vector<cudaEvent_t> free_events;
  double slot_ms[kNumSlots] = {};
  int64_t slot_launches[kNumSlots] = {};

  int per_step[kNumSlots] = {};  // kernels per slot per step for this box kind
  int64_t launches = 0;
  std::string err;
  bool poisoned = false;
};

namespace {

int fail(mpcd_t* h, int code, const std::string& msg) {
  if (h) {
    h->err = msg;
    if (code == MPCD_ERR_CUDA || code == MPCD_ERR_TIMEOUT) h->poisoned = true;
  } else {
    g_create_err = msg;
  }
  return code;
}

int cuda_fail(mpcd_t* h, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(h, e == cudaErrorMemoryAllocation ? MPCD_ERR_OOM : MPCD_ERR_CUDA, msg);
}

#define MPCD_TRY(h, call)                                    \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

bool is_pow2(double a) {
  int e;
  const double m = std::frexp(a, &e);
  return m == 0.5;
}

int check_params(const mpcd_params* p, std::string* why) {
  if (!p) return *why = "params is NULL", MPCD_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (p->L[d] < 1) return *why = "L must be >= 1 in every direction", MPCD_ERR_ARG;
  if (p->precision != MPCD_FP64 && p->precision != MPCD_MIXED) return *why = "unknown precision", MPCD_ERR_ARG;
  if (!(p->a > 0.0) || !std::isfinite(p->a)) return *why = "a must be > 0", MPCD_ERR_ARG;
  if (!(p->ppc >= 0.0) || !std::isfinite(p->ppc)) return *why = "ppc must be >= 0", MPCD_ERR_ARG;
  if (!(p->dt >= 0.0) || !std::isfinite(p->dt)) return *why = "dt must be >= 0", MPCD_ERR_ARG;
  if (!std::isfinite(p->alpha)) return *why = "alpha must be finite", MPCD_ERR_ARG;
  if (!(p->kT > 0.0) || !std::isfinite(p->kT)) return *why = "kT must be > 0", MPCD_ERR_ARG;
  if (!(p->mass > 0.0) || !std::isfinite(p->mass)) return *why = "mass must be > 0", MPCD_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(p->g[d])) return *why = "g must be finite", MPCD_ERR_ARG;
  if (p->walls_z != 0 && p->walls_z != 1) return *why = "walls_z must be 0 or 1", MPCD_ERR_ARG;
  if (p->walls_z && p->g[2] != 0.0) return *why = "g[2] must be 0 with walls in z", MPCD_ERR_ARG;
  if (p->thermostat < 0 || p->thermostat > 2) return *why = "thermostat must be 0, 1 or 2", MPCD_ERR_ARG;
  if (p->resort_k < 0) return *why = "resort_k must be >= 0", MPCD_ERR_ARG;
  if (p->angular != 0 && p->angular != 1) return *why = "angular must be 0 or 1", MPCD_ERR_ARG;
  if (p->angular && p->walls_z) return *why = "angular-momentum conservation needs a periodic box (no walls)", MPCD_ERR_ARG;
  if (p->precision == MPCD_MIXED) {
    int bits = 0;
    for (int d = 0; d < 3; ++d) {
      int b = 0;
      while ((1 << b) < p->L[d]) ++b;
      bits += b;
    }
    if (bits > 31) return *why = "mixed precision packs the cell coordinates in 31 bits: box too large", MPCD_ERR_ARG;
  }
  const double cells = (double)p->L[0] * p->L[1] * ((double)p->L[2] + (p->walls_z ? 1 : 0));
  if (cells > 2.0e9) return *why = "too many cells (limit 2e9)", MPCD_ERR_ARG;
  const double n = std::round(p->ppc * (double)p->L[0] * p->L[1] * p->L[2]);
  if (n > 2.0e9) return *why = "too many particles (limit 2e9)", MPCD_ERR_ARG;
  return MPCD_OK;
}

Geom make_geom(const mpcd_params* p) {
  Geom g{};
  for (int d = 0; d < 3; ++d) g.L[d] = p->L[d];
  g.walls = p->walls_z;
  g.thermostat = p->thermostat;
  g.angular = p->angular;
  g.resort_k = p->resort_k;
  g.a = p->a;
  g.inv_a = 1.0 / p->a;
  g.pow2a = is_pow2(p->a) ? 1 : 0;
  {
    int e2 = 0;
    std::frexp(p->a, &e2);
    g.log2a = g.pow2a ? e2 - 1 : 0;
  }
  for (int d = 0; d < 3; ++d) g.B[d] = (double)p->L[d] * p->a;
  g.dt = p->dt;
  g.force = 0;
  for (int d = 0; d < 3; ++d) {
    g.g[d] = p->g[d];
    g.h[d] = ((0.5 * p->g[d]) * p->dt) * p->dt;
    if (p->g[d] != 0.0) g.force = 1;
  }
  g.cos_a = std::cos(p->alpha);
  g.sin_a = std::sin(p->alpha);
  g.mass = p->mass;
  g.kT = p->kT;
  g.ppc = p->ppc;
  g.seed = p->seed;
  g.dta = static_cast<float>(p->dt / p->a);
  for (int d = 0; d < 3; ++d) {
    g.ha[d] = static_cast<float>(0.5 * p->g[d] * p->dt * p->dt / p->a);
    g.gdt[d] = static_cast<float>(p->g[d] * p->dt);
    int b = 0;
    while ((1 << b) < p->L[d]) ++b;
    g.bits[d] = b;
  }
  g.cos_af = static_cast<float>(g.cos_a);
  g.sin_af = static_cast<float>(g.sin_a);
  g.dtf = static_cast<float>(g.dt);
  g.inv_af = static_cast<float>(g.inv_a);
  for (int d = 0; d < 3; ++d) g.gf[d] = p->g[d] != 0.0 ? static_cast<float>(p->g[d]) : 0.0f;
  g.kTf = static_cast<float>(p->kT);
  g.massf = static_cast<float>(p->mass);
  g.n = (int64_t)std::llround(p->ppc * (double)p->L[0] * p->L[1] * p->L[2]);
  g.ncell = (int64_t)p->L[0] * p->L[1] * ((int64_t)p->L[2] + (p->walls_z ? 1 : 0));
  return g;
}

template <typename T>
int dalloc(mpcd_t* h, T** out, int64_t count) {
  void* p = nullptr;
  const size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(h, e, "cudaMalloc");
  }
  h->allocations.push_back(p);
  *out = static_cast<T*>(p);
  return MPCD_OK;
}

bool resort_at(const mpcd_t* h, int64_t t1) { return h->geom.resort_k > 0 && (t1 % h->geom.resort_k) == 0; }

cudaEvent_t get_event(mpcd_t* h) {
  if (!h->free_events.empty()) {
    cudaEvent_t e = h->free_events.back();
    h->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch one slot's kernels, bracketed by events when timing.
template <typename F>
int run_slot(mpcd_t* h, int slot, F&& launch) {
  PendingTiming pt{slot, nullptr, nullptr};
  if (h->timing) {
    pt.a = get_event(h);
    pt.b = get_event(h);
    MPCD_TRY(h, cudaEventRecord(pt.a, h->stream));
  }
  launch();
  MPCD_TRY(h, cudaGetLastError());
  if (h->timing) {
    MPCD_TRY(h, cudaEventRecord(pt.b, h->stream));
    h->pending.push_back(pt);
  }
  return MPCD_OK;
}

bool dense_fp64(const mpcd_t* h) { return h->precision == MPCD_FP64 && fp64_dense_collide(h->geom, h->scr); }

// The mixed form runs its staged path as one persistent launch per step (tuning fuse = 1).
bool one_launch_mixed(const mpcd_t* h) {
  return h->precision == MPCD_MIXED && h->tune.fuse && !h->mb.angular && !h->masses;
}

// Enqueue one piece of a step on h->stream.  `par` is the mixed form's buffer set at the start
// of the step (the FP64 kernels read theirs from the control block).
int enqueue_piece(mpcd_t* h, int piece, bool moments, int par = 0) {
  const Geom& g = h->geom;
  int rc;
  if (h->precision == MPCD_MIXED) {
    MixScratch m = h->mscr;
    const int nx = par ^ 1;
    if (one_launch_mixed(h)) {
      cudaError_t le = cudaSuccess;
      if ((rc = run_slot(h, kSlotStep, [&] {
             le = launch_step_mixed(h->mb, h->mix, m, h->ctl, moments, h->d_gspec, h->d_groups, h->d_bar,
                                    h->stall_test, h->stream);
           })))
        return rc;
      if (le != cudaSuccess) return cuda_fail(h, le, "one-launch step");
      return MPCD_OK;
    }
    if ((rc = run_slot(h, kSlotZero, [&] { launch_zero_i32_pair(m.count[nx], m.cursor, g.ncell, h->stream); })))
      return rc;
    if ((rc = run_slot(h, kSlotScan, [&] { launch_scan(m.count[par], m.offset, m.partial, g.ncell, h->stream); })))
      return rc;
    if ((rc = run_slot(h, kSlotScatter, [&] {
           launch_scatter_cursor(g.n, m.key[par], m.offset, m.cursor, m.perm, h->stream);
           launch_group_bounds(h->mb, h->d_gspec, m.offset, h->d_groups, h->stream);
         })))
      return rc;
    if ((rc = run_slot(h, kSlotCollide,
                       [&] { launch_collide_stream_mixed(h->mb, h->mix, m, h->ctl, moments, h->stream, h->mixm); })))
      return rc;
    if ((rc = run_slot(h, kSlotEndStep, [&] { launch_end_step_mixed(h->mb, h->ctl, h->stream); }))) return rc;
    return MPCD_OK;
  }
  Scratch s = h->scr;
  if (piece == kPieceTail)
    return run_slot(h, kSlotRotate, [&] { launch_rotate_fp64(g, h->f64, s, h->ctl, h->stream, h->f64m); });
  if (piece == kPieceStep) {
    if ((rc = enqueue_piece(h, kPieceFull, moments, par))) return rc;
    return enqueue_piece(h, kPieceTail, moments, par);
  }
  if ((rc = run_slot(h, kSlotZero, [&] { launch_zero_i32_pair(s.count, s.cursor, g.ncell, h->stream); }))) return rc;
  if (piece == kPieceBody) {
    if ((rc = run_slot(h, kSlotRotateStream,
                       [&] { launch_rotate_stream_fp64(g, h->f64, s, h->ctl, h->stream, h->f64m); })))
      return rc;
  } else {
    if ((rc = run_slot(h, kSlotStreamBin, [&] { launch_stream_bin_fp64(g, h->f64, s, h->ctl, h->stream); }))) return rc;
  }
  if ((rc = run_slot(h, kSlotScan, [&] { launch_scan(s.count, s.offset, s.partial, g.ncell, h->stream); }))) return rc;
  if ((rc = run_slot(h, kSlotScatter, [&] { launch_scatter(g, s, h->ctl, h->stream); }))) return rc;
  if ((rc = run_slot(h, kSlotCollide, [&] { launch_collide_fp64(g, h->f64, s, h->ctl, moments, h->stream, h->f64m); }))) return rc;
  if ((rc = run_slot(h, kSlotEndStep, [&] { launch_end_step(g, h->ctl, h->stream); }))) return rc;
  return MPCD_OK;
}

// Mixed form: keys, ranks and counts for the first step after the state was set.
int enqueue_bin_mixed(mpcd_t* h) {
  const Geom& g = h->geom;
  MixScratch m = h->mscr;
  const int par = h->cur;
  int rc;
  if ((rc = run_slot(h, kSlotZero, [&] { launch_zero_i32(m.count[par], g.ncell, h->stream); }))) return rc;
  if ((rc = run_slot(h, kSlotStreamBin, [&] { launch_bin_mixed(h->mb, h->mix, m, h->ctl, h->stream); }))) return rc;
  h->launches += 2;
  h->mixed_keys_valid = true;
  return MPCD_OK;
}

int piece_launches(const mpcd_t* h, int piece) {
  if (one_launch_mixed(h)) return 1;
  if (piece == kPieceTail) return h->per_step[kSlotRotate];
  if (piece == kPieceStep) return piece_launches(h, kPieceFull) + piece_launches(h, kPieceTail);
  int k = 0;
  for (int s = 0; s < kNumSlots; ++s) {
    if (s == kSlotRotate || s == kSlotStep || (s == kSlotRotateStream && piece != kPieceBody) ||
        (s == kSlotStreamBin && piece == kPieceBody))
      continue;
    k += h->per_step[s];
  }
  return k;
}

void drop_graph(mpcd_t* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  if (h->graph_body) cudaGraphExecDestroy(h->graph_body);
  h->graph_body = nullptr;
  if (h->graph_step) cudaGraphExecDestroy(h->graph_step);
  h->graph_step = nullptr;
  for (int k = 0; k < 2; ++k) {
    if (h->graph_par[k]) cudaGraphExecDestroy(h->graph_par[k]);
    h->graph_par[k] = nullptr;
  }
}

int capture_step(mpcd_t* h, int piece, int par, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  MPCD_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  const bool saved = h->timing;
  h->timing = false;
  int rc = enqueue_piece(h, piece, h->record_moments, par);
  h->timing = saved;
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
  return MPCD_OK;
}

int build_graph(mpcd_t* h) {
  drop_graph(h);
  int rc;
  if (h->precision == MPCD_MIXED) {
    for (int k = 0; k < 2; ++k)
      if ((rc = capture_step(h, kPieceFull, k, &h->graph_par[k]))) return rc;
  } else {
    if ((rc = capture_step(h, kPieceFull, 0, &h->graph))) return rc;
    if (dense_fp64(h) && (rc = capture_step(h, kPieceBody, 0, &h->graph_body))) return rc;
    if (dense_fp64(h) && (rc = capture_step(h, kPieceStep, 0, &h->graph_step))) return rc;
  }
  h->graph_moments = h->record_moments;
  return MPCD_OK;
}

// FP64 form: the state just written to buffer set 0 in particle-id order is put into cell
// order (unshifted grid, stable by slot) in buffer set 1, which becomes the current set, so
// that the first steps already read each cell's members from neighbouring slots.  The
// caller writes the control block afterwards with cur = h->cur.
int presort_fp64(mpcd_t* h) {
  h->cur = 0;
  if (h->precision != MPCD_FP64 || h->n == 0) return MPCD_OK;
  h->launches += launch_presort_fp64(h->geom, h->f64, h->scr, h->f64m, h->stream);
  MPCD_TRY(h, cudaGetLastError());
  h->cur = 1;
  return MPCD_OK;
}

int guard(mpcd_t* h) {
  if (!h) return MPCD_ERR_ARG;
  if (h->poisoned) return MPCD_ERR_STATE;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  return MPCD_OK;
}

// Mixed form: per-box grid shifts of steps t + 1 and t + 2 to the device.
int upload_shifts(mpcd_t* h, int64_t t) {
  std::vector<BoxShift> sh(h->boxes.size());
  for (size_t b = 0; b < h->boxes.size(); ++b) mixed_box_shifts(h->boxes[b], t, &sh[b]);
  MPCD_TRY(h, cudaMemcpyAsync(h->d_shifts, sh.data(), sizeof(BoxShift) * sh.size(), cudaMemcpyHostToDevice, h->stream));
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  return MPCD_OK;
}

// Mixed form: the table of warp groups (consecutive cells of one box, about
// tune.group_target particles each) for the current tuning.
int build_groups(mpcd_t* h) {
  // the fixed part of the group table: per box, ceil(N_b / T_b) groups of T_b records, with
  // T_b the target, at most 24 cells' worth on average (so groups rarely exceed 32 cells) and
  // at most the stage's kMixCap records less a high quantile of one cell's occupancy
  // (ppc + 4 sqrt(ppc)): a group overshoots its target by up to one cell, and a group past
  // kMixCap takes the slower per-cell path.  k_group_bounds places the cell boundaries
  // every step.
  std::vector<MixGroupSpec> spec;
  for (size_t b = 0; b < h->boxes.size(); ++b) {
    const Geom& g = h->boxes[b];
    const int64_t nb = h->pbase[b + 1] - h->pbase[b];
    const int64_t room = kMixCap - static_cast<int64_t>(std::ceil(g.ppc + 4.0 * std::sqrt(g.ppc)));
    const int64_t tb = std::max<int64_t>(
        16, std::min<int64_t>({static_cast<int64_t>(h->tune.group_target), static_cast<int64_t>(24.0 * g.ppc), room}));
    const int64_t ng = std::max<int64_t>(1, (nb + tb - 1) / tb);
    for (int64_t k = 0; k < ng; ++k) {
      MixGroupSpec x;
      x.rec0 = h->pbase[b] + k * tb;
      x.rec1 = k + 1 < ng ? h->pbase[b] + (k + 1) * tb : -1;
      x.box = static_cast<int32_t>(b);
      x.pad = 0;
      spec.push_back(x);
    }
  }
  if ((int64_t)spec.size() > 2000000000LL) return fail(h, MPCD_ERR_ARG, "too many cell groups");
  if ((int64_t)spec.size() > h->groups_cap) {
    for (void* p : {static_cast<void*>(h->d_groups), static_cast<void*>(h->d_gspec)}) {
      if (!p) continue;
      cudaFree(p);
      for (auto& q : h->allocations)
        if (q == p) q = nullptr;
    }
    h->d_groups = nullptr;
    h->d_gspec = nullptr;
    int rc = dalloc(h, &h->d_groups, (int64_t)spec.size());
    if (!rc) rc = dalloc(h, &h->d_gspec, (int64_t)spec.size());
    if (rc) return rc;
    h->groups_cap = (int64_t)spec.size();
  }
  MPCD_TRY(h, cudaMemcpyAsync(h->d_gspec, spec.data(), sizeof(MixGroupSpec) * spec.size(), cudaMemcpyHostToDevice,
                              h->stream));
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  h->mb.groups = h->d_groups;
  h->mb.ngroups = static_cast<int32_t>(spec.size());
  h->mb.warps = h->tune.warps;
  drop_graph(h);  // the graphs hold the old table
  return MPCD_OK;
}

int create_common(const mpcd_params* p, int32_t nbox, mpcd_t** out) {
  std::string why;
  for (int32_t b = 0; b < nbox; ++b) {
    int rc = check_params(&p[b], &why);
    if (rc) return fail(nullptr, rc, nbox > 1 ? "box " + std::to_string(b) + ": " + why : why);
  }
  if (nbox > 1) {
    for (int32_t b = 0; b < nbox; ++b) {
      if (p[b].precision != MPCD_MIXED) return fail(nullptr, MPCD_ERR_ARG, "ensembles use the mixed form (MPCD_MIXED)");
      if (p[b].walls_z != p[0].walls_z || p[b].thermostat != p[0].thermostat || p[b].angular != p[0].angular)
        return fail(nullptr, MPCD_ERR_ARG, "all boxes of an ensemble must share walls_z, thermostat and angular");
    }
  }
  mpcd_t* h = new mpcd_t();
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, MPCD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  h->precision = p[0].precision;
  h->nbox = nbox;
  h->tune.group_target = 168;
  h->tune.warps = 4;
  h->tune.resort_k = p[0].resort_k;
  // FP64: the fused rotate-and-stream pass is faster; mixed: the eight-launch step is (its
  // sort phases run at full occupancy), the one-launch step remains a tuning choice
  h->tune.fuse = p[0].precision == MPCD_FP64 ? 1 : 0;
  // per-box geometry; the handle's geom describes the whole concatenation for the kernels
  // that run over all cells or particles (zeroing, scan, sort)
  int64_t ctot = 0, ntot = 0;
  bool force = false;
  h->pbase.push_back(0);
  for (int32_t b = 0; b < nbox; ++b) {
    Geom g = make_geom(&p[b]);
    g.cbase = ctot;
    g.pbase = ntot;
    ctot += g.ncell;
    ntot += g.n;
    force = force || g.force;
    h->boxes.push_back(g);
    h->pbase.push_back(ntot);
  }
  if (ctot > 2000000000LL || ntot > 2000000000LL) {
    delete h;
    return fail(nullptr, MPCD_ERR_ARG, "the ensemble has more than 2e9 cells or particles");
  }
  h->geom = h->boxes[0];
  h->geom.n = ntot;
  h->geom.ncell = ctot;
  for (int k = 0; k < kNumSlots; ++k) h->per_step[k] = kSlotLaunchesBase[k];
  h->per_step[kSlotZero] = 1;  // counts and the scatter's cursors, one launch
  if (!h->geom.walls && !h->geom.thermostat) h->per_step[kSlotRotate] = h->per_step[kSlotRotateStream] = 1;
  h->n = ntot;
  h->ncell = ctot;
  auto bail = [&](int code) {
    std::string msg = h->err;
    mpcd_destroy(h);
    *out = nullptr;
    return fail(nullptr, code, msg);
  };
  int rc;
  if ((e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail(h, e, "cudaStreamCreate"));
  h->stream = h->own_stream;
  const int64_t n = h->n, C = h->ncell;
  if (h->precision == MPCD_MIXED) {
    if ((e = prepare_collide_mixed()) != cudaSuccess) return bail(cuda_fail(h, e, "collide kernel setup"));
    h->per_step[kSlotStreamBin] = 0;  // binning is fused into the collide kernel
    h->per_step[kSlotZero] = 1;
    h->per_step[kSlotScatter] = 2;  // scatter + group bounds
    h->per_step[kSlotCollide] = 1;
    h->per_step[kSlotRotate] = h->per_step[kSlotRotateStream] = 0;
    h->per_step[kSlotStep] = 1;
    for (int k = 0; k < 2; ++k) {
      if ((rc = dalloc(h, &h->mix.rec[k], n))) return bail(rc);
      if ((rc = dalloc(h, &h->mscr.key[k], n))) return bail(rc);
      if ((rc = dalloc(h, &h->mscr.count[k], C))) return bail(rc);
    }
    if ((rc = dalloc(h, &h->mscr.cursor, C))) return bail(rc);
    if ((rc = dalloc(h, &h->mscr.perm, n))) return bail(rc);
    if ((rc = dalloc(h, &h->mscr.offset, C + 1))) return bail(rc);
    // tile sums of both scans: the three-kernel one and the one-launch step's (smaller tiles)
    if ((rc = dalloc(h, &h->mscr.partial, std::max<int64_t>(scan_tiles(C), step_scan_tiles(C)) + 1))) return bail(rc);
    if ((rc = dalloc(h, &h->d_boxes, nbox))) return bail(rc);
    if ((rc = dalloc(h, &h->d_shifts, nbox))) return bail(rc);
    if ((rc = dalloc(h, &h->d_pbase, (int64_t)nbox + 1))) return bail(rc);
    if ((e = cudaMemcpyAsync(h->d_boxes, h->boxes.data(), sizeof(Geom) * h->boxes.size(), cudaMemcpyHostToDevice,
                             h->stream)) != cudaSuccess)
      return bail(cuda_fail(h, e, "cudaMemcpyAsync"));
    if ((e = cudaMemcpyAsync(h->d_pbase, h->pbase.data(), sizeof(int64_t) * h->pbase.size(), cudaMemcpyHostToDevice,
                             h->stream)) != cudaSuccess)
      return bail(cuda_fail(h, e, "cudaMemcpyAsync"));
    h->mb.boxes = h->d_boxes;
    h->mb.shifts = h->d_shifts;
    h->mb.pbase = h->d_pbase;
    h->mb.nbox = nbox;
    h->mb.n = n;
    h->mb.ncell = C;
    h->mb.walls = h->geom.walls;
    h->mb.force = force ? 1 : 0;
    h->mb.thermostat = h->geom.thermostat;
    h->mb.angular = h->geom.angular;
    if ((rc = build_groups(h))) return bail(rc);
    if ((rc = upload_shifts(h, 0))) return bail(rc);
  } else {
    for (int k = 0; k < 2; ++k) {  // one block per buffer set: r (3 n doubles), then v (3 n)
      double* set = nullptr;
      if ((rc = dalloc(h, &set, 6 * n))) return bail(rc);
      for (int d = 0; d < 3; ++d) {
        h->f64.r[k][d] = set + d * n;
        h->f64.v[k][d] = set + (3 + d) * n;
      }
      if ((rc = dalloc(h, &h->f64.id[k], n))) return bail(rc);
    }
    if ((rc = dalloc(h, &h->scr.key, n))) return bail(rc);
    h->scr.key2 = h->scr.key;
    if ((rc = dalloc(h, &h->scr.rank, n))) return bail(rc);
    if ((rc = dalloc(h, &h->scr.perm, n))) return bail(rc);
    if ((rc = dalloc(h, &h->scr.count, C))) return bail(rc);
    if ((rc = dalloc(h, &h->scr.cursor, C))) return bail(rc);
    if ((rc = dalloc(h, &h->scr.offset, C + 1))) return bail(rc);
    if ((rc = dalloc(h, &h->scr.partial, (int64_t)scan_tiles(C) + 1))) return bail(rc);
    if (!h->geom.walls && !h->geom.thermostat) {
      if ((rc = dalloc(h, &h->scr.frame, 16 * C))) return bail(rc);
      if ((rc = dalloc(h, &h->scr.key2, n))) return bail(rc);  // keys of odd steps (fused pass)
    }
  }
  if ((rc = dalloc(h, &h->ctl, 1))) return bail(rc);
  if ((rc = dalloc(h, &h->d_bad, 1))) return bail(rc);
  if ((rc = dalloc(h, &h->d_bar, 2))) return bail(rc);
  if ((e = cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream)) != cudaSuccess)
    return bail(cuda_fail(h, e, "cudaMemsetAsync"));
  h->red_blocks = 152 * 4;
  if ((rc = dalloc(h, &h->scr.red, 3 * (int64_t)h->red_blocks))) return bail(rc);
  h->ctl_host = Ctl{};
  set_shifts(h->geom, &h->ctl_host);
  if ((e = cudaMemcpyAsync(h->ctl, &h->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
    return bail(cuda_fail(h, e, "cudaMemcpyAsync"));
  if (h->precision == MPCD_MIXED) {
    for (const Geom& g : h->boxes) launch_init_mixed_box(g, h->mix, h->scr.red, h->red_blocks, h->ctl, h->stream);
  } else {
    launch_init_fp64(h->geom, h->f64, h->scr.red, h->red_blocks, h->ctl, h->stream);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(h, e, "init kernels"));
  if ((rc = presort_fp64(h))) return bail(rc);
  if (h->cur) {  // the presorted state is in buffer set 1 (the initial mean is no longer needed)
    h->ctl_host.cur = h->cur;
    if ((e = cudaMemcpyAsync(h->ctl, &h->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
      return bail(cuda_fail(h, e, "cudaMemcpyAsync"));
  }
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(cuda_fail(h, e, "init sync"));
  *out = h;
  return MPCD_OK;
}

}  // namespace

extern "C" {

int mpcd_create(const mpcd_params* p, mpcd_t** out) {
  if (!out) return fail(nullptr, MPCD_ERR_ARG, "out is NULL");
  *out = nullptr;
  return create_common(p, 1, out);
}

int mpcd_batch_create(int32_t nbox, const mpcd_params* p, mpcd_t** out) {
  if (!out) return fail(nullptr, MPCD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nbox < 1 || !p) return fail(nullptr, MPCD_ERR_ARG, "nbox must be >= 1 and params non-NULL");
  return create_common(p, nbox, out);
}

int mpcd_destroy(mpcd_t* h) {
  if (!h) return MPCD_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graph(h);
  for (auto& pt : h->pending) {
    cudaEventDestroy(pt.a);
    cudaEventDestroy(pt.b);
  }
  for (auto e : h->free_events) cudaEventDestroy(e);
  for (auto e : h->chunk_events) cudaEventDestroy(e);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  for (void* p : h->allocations) cudaFree(p);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
  return MPCD_OK;
}

int mpcd_set_stream(mpcd_t* h, void* stream) {
  int rc = guard(h);
  if (rc) return rc;
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  h->stream = stream ? static_cast<cudaStream_t>(stream) : h->own_stream;
  return MPCD_OK;
}

int mpcd_step(mpcd_t* h, int64_t nsteps) {
  int rc = guard(h);
  if (rc) return rc;
  if (nsteps < 0) return fail(h, MPCD_ERR_ARG, "nsteps must be >= 0");
  const bool mixed = h->precision == MPCD_MIXED;
  const bool dense = dense_fp64(h);
  const bool fused = dense && h->tune.fuse;
  for (int64_t k = 0; k < nsteps; ++k) {
    if (mixed && !h->mixed_keys_valid)
      if ((rc = enqueue_bin_mixed(h))) return rc;
    const int piece = !dense ? kPieceFull : !fused ? kPieceStep : (k > 0 ? kPieceBody : kPieceFull);
    if (h->timing) {
      if ((rc = enqueue_piece(h, piece, h->record_moments, h->cur))) return rc;
    } else {
      if ((mixed ? !h->graph_par[0] : !h->graph) || h->graph_moments != h->record_moments)
        if ((rc = build_graph(h))) return rc;
      cudaGraphExec_t ge = mixed ? h->graph_par[h->cur]
                                 : (piece == kPieceBody ? h->graph_body : piece == kPieceStep ? h->graph_step : h->graph);
      MPCD_TRY(h, cudaGraphLaunch(ge, h->stream));
    }
    h->launches += piece_launches(h, piece);
    h->t += 1;
    h->last_resorted = mixed || resort_at(h, h->t);
    if (h->last_resorted) h->cur ^= 1;
    h->perm_sorted = !mixed && (h->last_resorted || h->geom.walls || h->geom.thermostat || h->geom.angular);
    h->any_step = true;
    h->moments_valid = h->record_moments;
  }
  if (fused && nsteps > 0) {  // the last step's rotation
    if ((rc = enqueue_piece(h, kPieceTail, h->record_moments))) return rc;
    h->launches += piece_launches(h, kPieceTail);
  }
  return MPCD_OK;
}

// After a synchronisation: a bounded device-side wait that ran out (the one-launch mixed
// step's grid barriers) left its flag in the control block; the step is incomplete.
static int check_device_flag(mpcd_t* h) {
  if (h->precision != MPCD_MIXED) return MPCD_OK;
  int32_t err = 0;
  MPCD_TRY(h, cudaMemcpyAsync(&err, reinterpret_cast<const char*>(h->ctl) + offsetof(Ctl, err), sizeof(err),
                              cudaMemcpyDeviceToHost, h->stream));
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  if (err) return fail(h, MPCD_ERR_TIMEOUT, "a grid-wide barrier of the one-launch step waited too long; the step is incomplete");
  return MPCD_OK;
}

int mpcd_sync(mpcd_t* h) {
  int rc = guard(h);
  if (rc) return rc;
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  return check_device_flag(h);
}

int mpcd_debug_stall_barrier(mpcd_t* h, int32_t enable) {
  int rc = guard(h);
  if (rc) return rc;
  h->stall_test = enable ? 1 : 0;
  drop_graph(h);  // the captured step holds the flag
  return MPCD_OK;
}

int64_t mpcd_num_particles(const mpcd_t* h) { return h ? h->n : -1; }
int64_t mpcd_num_cells(const mpcd_t* h) { return h ? h->ncell : -1; }
int64_t mpcd_steps_done(const mpcd_t* h) { return h ? h->t : -1; }
int32_t mpcd_num_boxes(const mpcd_t* h) { return h ? h->nbox : -1; }

int mpcd_get_state_device(mpcd_t* h, double* r_dev, double* v_dev) {
  int rc = guard(h);
  if (rc) return rc;
  if (!r_dev || !v_dev) return fail(h, MPCD_ERR_ARG, "NULL output");
  if (h->precision == MPCD_MIXED)
    launch_get_state_mixed(h->mb, h->mix, h->cur, r_dev, v_dev, h->stream);
  else
    launch_get_state_fp64(h->geom, h->f64, h->cur, r_dev, v_dev, h->stream);
  MPCD_TRY(h, cudaGetLastError());
  h->launches += 1;
  return MPCD_OK;
}

int mpcd_set_masses(mpcd_t* h, int64_t n, const double* m) {
  int rc = guard(h);
  if (rc) return rc;
  const bool mixed = h->precision == MPCD_MIXED;
  if (n != h->n) return fail(h, MPCD_ERR_ARG, "n must equal mpcd_num_particles");
  if (!m) {
    h->masses = false;
    h->f64m.m[0] = h->f64m.m[1] = nullptr;
    h->mixm.m[0] = h->mixm.m[1] = nullptr;
  } else {
    if (mixed && h->geom.angular)
      return fail(h, MPCD_ERR_ARG,
                  "particle masses with angular-momentum conservation need the FP64 form (MPCD_FP64)");
    std::vector<double> m32;
    for (int64_t i = 0; i < n; ++i)
      if (!(m[i] > 0.0) || !std::isfinite(m[i]) || (mixed && !(static_cast<float>(m[i]) > 0.0f)) ||
          (mixed && !std::isfinite(static_cast<float>(m[i]))))
        return fail(h, MPCD_ERR_ARG, "masses must be finite and > 0 (particle " + std::to_string(i) + ")");
    if (mixed) {  // the mixed form keeps FP32 masses; get_masses reports those values
      m32.resize((size_t)n);
      for (int64_t i = 0; i < n; ++i) m32[(size_t)i] = static_cast<double>(static_cast<float>(m[i]));
      m = m32.data();
    }
    if (!h->mass_buf[2] && (rc = dalloc(h, &h->mass_buf[2], n > 0 ? n : 1))) return rc;
    for (int k = 0; k < 2; ++k) {
      if (!mixed && !h->mass_buf[k] && (rc = dalloc(h, &h->mass_buf[k], n > 0 ? n : 1))) return rc;
      if (mixed && !h->mix_mass_buf[k] && (rc = dalloc(h, &h->mix_mass_buf[k], n > 0 ? n : 1))) return rc;
    }
    MPCD_TRY(h, cudaMemcpyAsync(h->mass_buf[2], m, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    // into the storage order of the current buffer set; a re-sort carries them along
    if (mixed)
      launch_gather_masses_mixed(n, h->mix.rec[h->cur], h->mass_buf[2], h->mix_mass_buf[h->cur], h->stream);
    else
      launch_gather_masses(n, h->mass_buf[2], h->f64.id[h->cur], h->mass_buf[h->cur], h->stream);
    MPCD_TRY(h, cudaGetLastError());
    h->launches += 1;
    h->masses = true;
    if (mixed) {
      h->mixm.m[0] = h->mix_mass_buf[0];
      h->mixm.m[1] = h->mix_mass_buf[1];
    } else {
      h->f64m.m[0] = h->mass_buf[0];
      h->f64m.m[1] = h->mass_buf[1];
    }
  }
  if (!mixed) h->per_step[kSlotRotate] = h->per_step[kSlotRotateStream] = (!h->geom.walls && !h->geom.thermostat) ? 1 : 0;
  drop_graph(h);  // the step graph holds the buffer pointers and the kernel choice
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  return MPCD_OK;
}

int mpcd_get_masses(mpcd_t* h, double* m) {
  int rc = guard(h);
  if (rc) return rc;
  if (!m) return fail(h, MPCD_ERR_ARG, "NULL output");
  if (!h->masses) {
    for (int64_t i = 0; i < h->n; ++i) m[i] = h->geom.mass;
    return MPCD_OK;
  }
  MPCD_TRY(h, cudaMemcpyAsync(m, h->mass_buf[2], sizeof(double) * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream));
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  return MPCD_OK;
}

// The handle's staging buffer for host copies of the state (6 N doubles), allocated on the
// first host get/set_state and kept: a stream-ordered allocation per call would map and
// release it again at every synchronisation.
static int host_stage(mpcd_t* h, double** out) {
  if (!h->host_stage) {
    int rc = dalloc(h, &h->host_stage, 6 * (h->n > 0 ? h->n : 1));
    if (rc) return rc;
  }
  *out = h->host_stage;
  return MPCD_OK;
}

int mpcd_get_state(mpcd_t* h, double* r, double* v) {
  int rc = guard(h);
  if (rc) return rc;
  if (!r || !v) return fail(h, MPCD_ERR_ARG, "NULL output");
  // gather into the staging buffer, then copy to the host
  double* scratch = nullptr;
  if ((rc = host_stage(h, &scratch))) return rc;
  constexpr int kChunks = 8;
  if (h->precision == MPCD_FP64 && h->n >= 65536) {
    // by particle id in chunks: each chunk is gathered (contiguous writes) while the previous
    // one is copied to the host on a second stream
    if (!h->copy_stream) {
      MPCD_TRY(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
      h->chunk_events.assign(kChunks, nullptr);
      for (auto& ev : h->chunk_events) MPCD_TRY(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    const int64_t n = h->n;
    launch_slot_of(h->geom, h->f64, h->cur, h->scr.rank, h->stream);
    for (int c = 0; c < kChunks; ++c) {
      const int64_t p0 = n * c / kChunks, p1 = n * (c + 1) / kChunks;
      launch_gather_by_id(p0, p1, h->scr.rank, h->f64, h->cur, scratch, scratch + 3 * n, h->stream);
      MPCD_TRY(h, cudaGetLastError());
      MPCD_TRY(h, cudaEventRecord(h->chunk_events[c], h->stream));
      MPCD_TRY(h, cudaStreamWaitEvent(h->copy_stream, h->chunk_events[c], 0));
      MPCD_TRY(h, cudaMemcpyAsync(r + 3 * p0, scratch + 3 * p0, sizeof(double) * 3 * (size_t)(p1 - p0),
                                  cudaMemcpyDeviceToHost, h->copy_stream));
      MPCD_TRY(h, cudaMemcpyAsync(v + 3 * p0, scratch + 3 * n + 3 * p0, sizeof(double) * 3 * (size_t)(p1 - p0),
                                  cudaMemcpyDeviceToHost, h->copy_stream));
    }
    MPCD_TRY(h, cudaStreamSynchronize(h->copy_stream));
    MPCD_TRY(h, cudaStreamSynchronize(h->stream));
    h->launches += 1 + kChunks;
    return MPCD_OK;
  }
  if (h->precision == MPCD_MIXED)
    launch_get_state_mixed(h->mb, h->mix, h->cur, scratch, scratch + 3 * h->n, h->stream);
  else
    launch_get_state_fp64(h->geom, h->f64, h->cur, scratch, scratch + 3 * h->n, h->stream);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(r, scratch, sizeof(double) * 3 * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(v, scratch + 3 * h->n, sizeof(double) * 3 * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_state");
  h->launches += 1;
  return check_device_flag(h);
}

// Reject a state with a position outside its box or a non-finite velocity before any of it
// is applied (checked on the device; synchronises).
static int check_state(mpcd_t* h, const double* r_dev, const double* v_dev) {
  MPCD_TRY(h, cudaMemsetAsync(h->d_bad, 0xFF, sizeof(unsigned long long), h->stream));
  launch_check_state(h->precision == MPCD_MIXED ? &h->mb : nullptr, h->geom, h->n, r_dev, v_dev, h->d_bad, h->stream);
  MPCD_TRY(h, cudaGetLastError());
  unsigned long long bad = 0;
  MPCD_TRY(h, cudaMemcpyAsync(&bad, h->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  if (bad != ~0ull)
    return fail(h, MPCD_ERR_ARG, "position outside its box or non-finite velocity at particle " + std::to_string(bad));
  return MPCD_OK;
}

// Apply a checked state.  FP64: straight into cell order (the initial sort, R25) in buffer
// set 1, masses along; gathered >= 0: the state already stands in cell order in that buffer
// set (the overlapped host upload), which becomes the current one.
static int apply_state(mpcd_t* h, int64_t n, const double* r_dev, const double* v_dev, int64_t t, int gathered) {
  int rc = MPCD_OK;
  h->cur = 0;
  if (gathered >= 0) {
    h->cur = gathered;
  } else if (h->precision == MPCD_MIXED) {
    launch_set_state_mixed(h->mb, h->mix, r_dev, v_dev, h->stream);
    if (h->masses)  // the new records are in particle-id order
      launch_gather_masses_mixed(n, h->mix.rec[0], h->mass_buf[2], h->mix_mass_buf[0], h->stream);
  } else if (n > 0) {
    const double* m_by_id = h->masses ? h->mass_buf[2] : nullptr;
    double* m_dst = h->masses ? h->mass_buf[1] : nullptr;
    h->launches += launch_set_state_sorted_fp64(h->geom, h->f64, h->scr, r_dev, v_dev, m_by_id, m_dst, h->stream);
    h->cur = 1;
  }
  MPCD_TRY(h, cudaGetLastError());
  h->mixed_keys_valid = false;
  h->ctl_host = Ctl{};
  h->ctl_host.t = t;
  h->ctl_host.cur = h->cur;
  set_shifts(h->geom, &h->ctl_host);
  MPCD_TRY(h, cudaMemcpyAsync(h->ctl, &h->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream));
  if (h->precision == MPCD_MIXED)
    if ((rc = upload_shifts(h, t))) return rc;
  h->launches += 1;
  h->t = t;
  h->any_step = false;
  h->last_resorted = false;
  h->moments_valid = false;
  return MPCD_OK;
}

int mpcd_set_state_device(mpcd_t* h, int64_t n, const double* r_dev, const double* v_dev, int64_t t) {
  int rc = guard(h);
  if (rc) return rc;
  if (n != h->n) return fail(h, MPCD_ERR_ARG, "n must equal mpcd_num_particles");
  if (!r_dev || !v_dev || t < 0) return fail(h, MPCD_ERR_ARG, "NULL input or negative t");
  if ((rc = check_state(h, r_dev, v_dev))) return rc;
  return apply_state(h, n, r_dev, v_dev, t, -1);
}

// FP64 host upload of a large state, gathered into the buffer set that does not hold the
// current state: the positions go first, and their check, the whole cell-order sort and their
// gather run on the second stream while the velocities are still being copied; the
// velocities are checked and gathered on arrival.  One synchronisation at the end: a state
// that failed a check is never made current, so the current one stays as it was.
static int set_state_overlapped(mpcd_t* h, int64_t n, const double* r, const double* v, int64_t t,
                                double* scratch) {
  if (!h->copy_stream) {
    MPCD_TRY(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    h->chunk_events.assign(8, nullptr);
    for (auto& ev : h->chunk_events) MPCD_TRY(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  const int target = h->cur ^ 1;
  const double* m_by_id = h->masses ? h->mass_buf[2] : nullptr;
  double* m_dst = h->masses ? h->mass_buf[target] : nullptr;
  double* r_dev = scratch;
  double* v_dev = scratch + 3 * n;
  MPCD_TRY(h, cudaMemsetAsync(h->d_bad, 0xFF, sizeof(unsigned long long), h->stream));
  MPCD_TRY(h, cudaMemcpyAsync(r_dev, r, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
  MPCD_TRY(h, cudaEventRecord(h->chunk_events[0], h->stream));
  MPCD_TRY(h, cudaMemcpyAsync(v_dev, v, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
  MPCD_TRY(h, cudaStreamWaitEvent(h->copy_stream, h->chunk_events[0], 0));
  launch_check_positions(h->geom, n, r_dev, h->d_bad, h->copy_stream);
  h->launches += 1 + launch_sort_positions_fp64(h->geom, h->scr, r_dev, h->copy_stream);
  MPCD_TRY(h, cudaEventRecord(h->chunk_events[1], h->copy_stream));  // perm is ready
  h->launches += launch_gather_positions_fp64(h->geom, h->f64, h->scr, r_dev, target, h->copy_stream);
  MPCD_TRY(h, cudaGetLastError());
  MPCD_TRY(h, cudaEventRecord(h->chunk_events[2], h->copy_stream));
  launch_check_velocities(n, v_dev, h->d_bad, h->stream);
  MPCD_TRY(h, cudaStreamWaitEvent(h->stream, h->chunk_events[1], 0));
  h->launches += 1 + launch_gather_velocities_fp64(h->geom, h->f64, h->scr, v_dev, target, m_by_id, m_dst, h->stream);
  MPCD_TRY(h, cudaGetLastError());
  MPCD_TRY(h, cudaStreamWaitEvent(h->stream, h->chunk_events[2], 0));
  unsigned long long bad = 0;
  MPCD_TRY(h, cudaMemcpyAsync(&bad, h->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  if (bad != ~0ull) {
    h->any_step = false;  // the last step's sort record was overwritten by this one
    return fail(h, MPCD_ERR_ARG, "position outside its box or non-finite velocity at particle " + std::to_string(bad));
  }
  int rc = apply_state(h, n, r_dev, v_dev, t, target);
  if (rc) return rc;
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  return MPCD_OK;
}

int mpcd_set_state(mpcd_t* h, int64_t n, const double* r, const double* v, int64_t t) {
  int rc = guard(h);
  if (rc) return rc;
  if (n != h->n) return fail(h, MPCD_ERR_ARG, "n must equal mpcd_num_particles");
  if (!r || !v || t < 0) return fail(h, MPCD_ERR_ARG, "NULL input or negative t");
  double* scratch = nullptr;  // the state is uploaded, then checked and applied on the device
  if ((rc = host_stage(h, &scratch))) return rc;
  if (h->precision == MPCD_FP64 && n >= 65536) return set_state_overlapped(h, n, r, v, t, scratch);
  cudaError_t e = cudaMemcpyAsync(scratch, r, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(scratch + 3 * n, v, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_state copy");
  rc = mpcd_set_state_device(h, n, scratch, scratch + 3 * n, t);
  if (rc) return rc;
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  return MPCD_OK;
}

int mpcd_add_momentum_device(mpcd_t* h, int64_t n, const double* dp_dev) {
  int rc = guard(h);
  if (rc) return rc;
  if (n != h->n) return fail(h, MPCD_ERR_ARG, "n must equal mpcd_num_particles");
  if (!dp_dev && n > 0) return fail(h, MPCD_ERR_ARG, "NULL input");
  if (h->precision == MPCD_MIXED)
    launch_add_momentum_mixed(h->mb, h->mix, h->cur, h->mixm, dp_dev, h->stream);
  else
    launch_add_momentum_fp64(h->geom, h->f64, h->cur, h->f64m, dp_dev, h->stream);
  MPCD_TRY(h, cudaGetLastError());
  h->launches += 1;
  return MPCD_OK;
}

int mpcd_add_momentum(mpcd_t* h, int64_t n, const double* dp) {
  int rc = guard(h);
  if (rc) return rc;
  if (n != h->n) return fail(h, MPCD_ERR_ARG, "n must equal mpcd_num_particles");
  if (!dp && n > 0) return fail(h, MPCD_ERR_ARG, "NULL input");
  double* scratch = nullptr;  // the increments are uploaded into the staging buffer
  if ((rc = host_stage(h, &scratch))) return rc;
  MPCD_TRY(h, cudaMemcpyAsync(scratch, dp, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
  if ((rc = mpcd_add_momentum_device(h, n, scratch))) return rc;
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));  // the staging buffer is reused by the next host call
  return MPCD_OK;
}

int mpcd_record_moments(mpcd_t* h, int32_t enable) {
  int rc = guard(h);
  if (rc) return rc;
  if (enable && !h->scr.moments) {
    if ((rc = dalloc(h, &h->scr.moments, 5 * h->ncell))) return rc;
    h->mscr.moments = h->scr.moments;
  }
  h->record_moments = enable != 0;
  h->moments_valid = false;
  return MPCD_OK;
}

int mpcd_cell_moments(mpcd_t* h, double* out, double* shift_out) {
  int rc = guard(h);
  if (rc) return rc;
  if (!out) return fail(h, MPCD_ERR_ARG, "NULL output");
  if (!h->moments_valid) return fail(h, MPCD_ERR_STATE, "no step has recorded moments (call mpcd_record_moments first)");
  MPCD_TRY(h, cudaMemcpyAsync(out, h->scr.moments, sizeof(double) * 5 * (size_t)h->ncell, cudaMemcpyDeviceToHost, h->stream));
  Ctl c{};
  MPCD_TRY(h, cudaMemcpyAsync(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  if (shift_out) {
    if (h->precision == MPCD_MIXED) {
      BoxShift b0{};
      MPCD_TRY(h, cudaMemcpy(&b0, h->d_shifts, sizeof(BoxShift), cudaMemcpyDeviceToHost));
      for (int d = 0; d < 3; ++d) shift_out[d] = b0.s_last[d];
    } else {
      for (int d = 0; d < 3; ++d) shift_out[d] = c.shift_last[d];
    }
  }
  return MPCD_OK;
}

int mpcd_debug_sort(mpcd_t* h, int32_t* keys, int32_t* counts, int32_t* offsets, int32_t* perm, int32_t* ids) {
  int rc = guard(h);
  if (rc) return rc;
  if (!h->any_step) return fail(h, MPCD_ERR_STATE, "no step has run since the state was set");
  const bool mixed = h->precision == MPCD_MIXED;
  // the storage order at the start of the last step: the other buffer set after a re-sort
  const int before = h->last_resorted ? (h->cur ^ 1) : h->cur;
  Scratch s = h->scr;
  if (mixed) {
    s.key = h->mscr.key[before];
    s.count = h->mscr.count[before];
    s.offset = h->mscr.offset;
    s.perm = h->mscr.perm;
  }
  if (perm && !h->perm_sorted) {
    // ordinary steps leave each cell's entries in arrival order; sort them for the caller
    launch_sort_segments(h->geom, s, h->stream);
    MPCD_TRY(h, cudaGetLastError());
    h->launches += 1;
    h->perm_sorted = true;
  }
  const size_t nb = sizeof(int32_t) * (size_t)h->n, cb = sizeof(int32_t) * (size_t)h->ncell;
  const int32_t* keys_last = (!mixed && (h->t & 1)) ? s.key2 : s.key;  // keys of step h->t
  if (keys) MPCD_TRY(h, cudaMemcpyAsync(keys, keys_last, nb, cudaMemcpyDeviceToHost, h->stream));
  if (counts) MPCD_TRY(h, cudaMemcpyAsync(counts, s.count, cb, cudaMemcpyDeviceToHost, h->stream));
  if (offsets) MPCD_TRY(h, cudaMemcpyAsync(offsets, s.offset, cb + sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  if (perm) MPCD_TRY(h, cudaMemcpyAsync(perm, s.perm, nb, cudaMemcpyDeviceToHost, h->stream));
  if (ids) {
    if (mixed) {
      std::vector<MixRec> recs((size_t)h->n);
      MPCD_TRY(h, cudaMemcpyAsync(recs.data(), h->mix.rec[before], sizeof(MixRec) * (size_t)h->n,
                                  cudaMemcpyDeviceToHost, h->stream));
      MPCD_TRY(h, cudaStreamSynchronize(h->stream));
      for (int64_t i = 0; i < h->n; ++i) ids[i] = recs[(size_t)i].id;
    } else {
      MPCD_TRY(h, cudaMemcpyAsync(ids, h->f64.id[before], nb, cudaMemcpyDeviceToHost, h->stream));
    }
  }
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  return MPCD_OK;
}

int mpcd_timing(mpcd_t* h, int32_t enable) {
  int rc = guard(h);
  if (rc) return rc;
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  for (auto& pt : h->pending) {
    h->free_events.push_back(pt.a);
    h->free_events.push_back(pt.b);
  }
  h->pending.clear();
  for (int s = 0; s < kNumSlots; ++s) {
    h->slot_ms[s] = 0.0;
    h->slot_launches[s] = 0;
  }
  h->timing = enable != 0;
  return MPCD_OK;
}

int mpcd_timing_read(mpcd_t* h, int32_t nmax, const char** names, double* ms, int64_t* launches) {
  int rc = guard(h);
  if (rc) return rc;
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  for (auto& pt : h->pending) {
    float el = 0.f;
    MPCD_TRY(h, cudaEventElapsedTime(&el, pt.a, pt.b));
    h->slot_ms[pt.slot] += el;
    h->slot_launches[pt.slot] += h->per_step[pt.slot];
    h->free_events.push_back(pt.a);
    h->free_events.push_back(pt.b);
  }
  h->pending.clear();
  int k = 0;
  for (int s = 0; s < kNumSlots && k < nmax; ++s) {
    if (h->slot_launches[s] == 0) continue;
    if (names) names[k] = kSlotNames[s];
    if (ms) ms[k] = h->slot_ms[s];
    if (launches) launches[k] = h->slot_launches[s];
    ++k;
  }
  return k;
}

int64_t mpcd_launch_count(const mpcd_t* h) { return h ? h->launches : -1; }

int mpcd_box_offsets(const mpcd_t* h, int64_t* particle_base, int64_t* cell_base) {
  if (!h) return MPCD_ERR_ARG;
  const size_t nb = h->precision == MPCD_MIXED ? h->boxes.size() : 1;
  for (size_t b = 0; b <= nb; ++b) {
    if (particle_base) particle_base[b] = b < nb ? (h->precision == MPCD_MIXED ? h->boxes[b].pbase : 0) : h->n;
    if (cell_base) cell_base[b] = b < nb ? (h->precision == MPCD_MIXED ? h->boxes[b].cbase : 0) : h->ncell;
  }
  return MPCD_OK;
}

int mpcd_autotune(mpcd_t* h, int32_t trial_steps, mpcd_tuning* best, double* best_ms) {
  int rc = guard(h);
  if (rc) return rc;
  if (trial_steps < 1) return fail(h, MPCD_ERR_ARG, "trial_steps must be >= 1");
  if (h->timing) return fail(h, MPCD_ERR_STATE, "disable timing before autotuning");
  std::vector<mpcd_tuning> cand;
  if (h->precision == MPCD_MIXED) {
    for (int f : {1, 0})
      for (int w : {2, 4})
        for (int tg : {128, 144, 160, 168, 176}) cand.push_back(mpcd_tuning{tg, w, h->tune.resort_k, f});
  } else {
    for (int f : {0, 1})
      for (int k : {1, 2, 5, 10, 20, 50}) cand.push_back(mpcd_tuning{h->tune.group_target, h->tune.warps, k, f});
  }
  // keep the state: by-id FP64 copies are exact for both forms
  const int64_t t0 = h->t;
  double* save = nullptr;
  MPCD_TRY(h, cudaMallocAsync(reinterpret_cast<void**>(&save), sizeof(double) * 6 * (size_t)(h->n > 0 ? h->n : 1),
                              h->stream));
  if ((rc = mpcd_get_state_device(h, save, save + 3 * h->n))) return rc;
  cudaEvent_t ea = nullptr, eb = nullptr;
  MPCD_TRY(h, cudaEventCreate(&ea));
  MPCD_TRY(h, cudaEventCreate(&eb));
  double best_t = 1e300;
  mpcd_tuning choice = h->tune;
  for (const mpcd_tuning& c : cand) {
    if ((rc = mpcd_set_tuning(h, &c))) break;
    if ((rc = mpcd_step(h, 2))) break;  // builds the graph, warms the caches
    MPCD_TRY(h, cudaEventRecord(ea, h->stream));
    if ((rc = mpcd_step(h, trial_steps))) break;
    MPCD_TRY(h, cudaEventRecord(eb, h->stream));
    MPCD_TRY(h, cudaEventSynchronize(eb));
    float ms = 0.f;
    MPCD_TRY(h, cudaEventElapsedTime(&ms, ea, eb));
    const double per = (double)ms / trial_steps;
    if (per < best_t) {
      best_t = per;
      choice = c;
    }
  }
  cudaEventDestroy(ea);
  cudaEventDestroy(eb);
  if (!rc) rc = mpcd_set_tuning(h, &choice);
  if (!rc) rc = mpcd_set_state_device(h, h->n, save, save + 3 * h->n, t0);
  cudaFreeAsync(save, h->stream);
  if (rc) return rc;
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  if (best) *best = choice;
  if (best_ms) *best_ms = best_t;
  return MPCD_OK;
}

int mpcd_get_tuning(const mpcd_t* h, mpcd_tuning* out) {
  if (!h || !out) return MPCD_ERR_ARG;
  *out = h->tune;
  return MPCD_OK;
}

int mpcd_set_tuning(mpcd_t* h, const mpcd_tuning* t) {
  int rc = guard(h);
  if (rc) return rc;
  if (!t || (t->fuse != 0 && t->fuse != 1) || t->group_target < 32 || t->group_target > 224 ||
      (t->warps != 2 && t->warps != 4) || t->resort_k < 0)
    return fail(h, MPCD_ERR_ARG, "tuning out of range (group_target 32..224, warps 2 or 4, resort_k >= 0, fuse 0 or 1)");
  MPCD_TRY(h, cudaStreamSynchronize(h->stream));
  const mpcd_tuning old = h->tune;
  h->tune = *t;
  if (h->precision == MPCD_MIXED) {
    if (old.group_target != t->group_target || old.warps != t->warps) return build_groups(h);
    if (old.fuse != t->fuse) drop_graph(h);
  } else if (old.resort_k != t->resort_k || old.fuse != t->fuse) {
    // the re-sort schedule is part of the captured step and of the step-end kernel
    h->geom.resort_k = t->resort_k;
    drop_graph(h);
  }
  return MPCD_OK;
}

const char* mpcd_last_error(const mpcd_t* h) {
  if (h) return h->err.c_str();
  return g_create_err.c_str();
}

const char* mpcd_version(void) { return "libmpcd sm_103a"; }

}  // extern "C"

// ---- one FP64 step without any device allocation ----
//
// The sort scratch (cell keys, arrival ranks, permutation, counts, offsets, scan partials
// and the step control block) sits in a single file-scope device array.  Host code only
// ever sees the array's host-side stand-in symbol, so its device address is looked up once
// per device with cudaGetSymbolAddress and cached; kernels receive that address.
namespace {
constexpr int64_t kNaMaxParticles = MPCD_NOALLOC_MAX_PARTICLES;
constexpr int64_t kNaMaxCells = MPCD_NOALLOC_MAX_CELLS;
constexpr size_t kNaAlign = 256;
constexpr size_t na_round(size_t b) { return (b + kNaAlign - 1) / kNaAlign * kNaAlign; }
constexpr size_t kNaCtlBytes = na_round(sizeof(Ctl));
constexpr size_t kNaPartBytes = na_round(sizeof(int32_t) * (size_t)kNaMaxParticles);
constexpr size_t kNaCellBytes = na_round(sizeof(int32_t) * (size_t)(kNaMaxCells + 1));
constexpr size_t kNaScanBytes = na_round(sizeof(int32_t) * (size_t)(kNaMaxCells / 2048 + 2));
constexpr size_t kNaBytes = kNaCtlBytes + 3 * kNaPartBytes + 2 * kNaCellBytes + kNaScanBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
// Per device: the scratch array's device address and the id of the context it was looked
// up in.  A device reset (or any teardown of the primary context) loads the module again at
// another address, so the address is looked up again whenever the current context's id
// differs from the cached one.
unsigned char* g_na_ptr[kNaMaxDevices] = {};
unsigned long long g_na_ctx[kNaMaxDevices] = {};

// The current context's unique id through the driver API, reached by entry point so that
// the library needs no link against the driver library.  0 when it cannot be read.
unsigned long long current_context_id() {
  typedef CUresult (*GetCurrent)(CUcontext*);
  typedef CUresult (*GetId)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {  // callers hold g_na_mu
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
    looked_up = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

__global__ void k_noalloc_ctl(Geom g, Ctl* c, int64_t t) {
  c->t = t;
  c->cur = 0;
  c->err = 0;
  set_shifts(g, c);
}

int na_fail(int code, const std::string& msg) { return fail(nullptr, code, msg); }
}  // namespace

extern "C" int mpcd_step_fp64_noalloc(const mpcd_params* p, int64_t t, int64_t n, double* x, double* y, double* z,
                                      double* vx, double* vy, double* vz, void* stream) {
  std::string why;
  int rc = check_params(p, &why);
  if (rc) return na_fail(rc, why);
  if (p->precision != MPCD_FP64) return na_fail(MPCD_ERR_ARG, "mpcd_step_fp64_noalloc needs precision MPCD_FP64");
  if (t < 0 || n < 0) return na_fail(MPCD_ERR_ARG, "t and n must be >= 0");
  Geom g = make_geom(p);
  if (n > kNaMaxParticles)
    return na_fail(MPCD_ERR_ARG, "n = " + std::to_string(n) + " exceeds MPCD_NOALLOC_MAX_PARTICLES = " +
                                     std::to_string(kNaMaxParticles));
  if (g.ncell > kNaMaxCells)
    return na_fail(MPCD_ERR_ARG, "the box has " + std::to_string(g.ncell) + " cells, more than MPCD_NOALLOC_MAX_CELLS = " +
                                     std::to_string(kNaMaxCells));
  if (n > 0 && !(x && y && z && vx && vy && vz)) return na_fail(MPCD_ERR_ARG, "NULL particle array");
  // an error left pending by earlier work on this thread is not ours to report or clear
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "a CUDA error was already pending before mpcd_step_fp64_noalloc");
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= kNaMaxDevices) return na_fail(MPCD_ERR_ARG, "device index out of range");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_na_ptr[dev] || ctx == 0 || ctx != g_na_ctx[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress");
      g_na_ptr[dev] = static_cast<unsigned char*>(ptr);
      g_na_ctx[dev] = current_context_id();  // the lookup made the primary context current
    }
    base = g_na_ptr[dev];
  }
  g.n = n;
  g.resort_k = 0;  // storage order is the caller's and never changes
  Ctl* ctl = reinterpret_cast<Ctl*>(base);
  unsigned char* q = base + kNaCtlBytes;
  Scratch s{};
  s.key = reinterpret_cast<int32_t*>(q);
  s.key2 = s.key;
  q += kNaPartBytes;
  s.rank = reinterpret_cast<int32_t*>(q);
  q += kNaPartBytes;
  s.perm = reinterpret_cast<int32_t*>(q);
  q += kNaPartBytes;
  s.count = reinterpret_cast<int32_t*>(q);
  q += kNaCellBytes;
  s.offset = reinterpret_cast<int32_t*>(q);
  q += kNaCellBytes;
  s.partial = reinterpret_cast<int32_t*>(q);
  Fp64Bufs b{};
  b.r[0][0] = x;
  b.r[0][1] = y;
  b.r[0][2] = z;
  b.v[0][0] = vx;
  b.v[0][1] = vy;
  b.v[0][2] = vz;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_noalloc_ctl<<<1, 1, 0, st>>>(g, ctl, t);
  launch_zero_i32(s.count, g.ncell, st);
  launch_stream_bin_fp64(g, b, s, ctl, st);
  launch_scan(s.count, s.offset, s.partial, g.ncell, st);
  launch_scatter(g, s, ctl, st);
  launch_collide_fp64_generic(g, b, s, ctl, false, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "mpcd_step_fp64_noalloc launch");
  return MPCD_OK;
}
