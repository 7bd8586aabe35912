// bpm.cu - host side of libbpm.so: plans, launches and the C ABI of bpm.h.
//
// Plans validate problem descriptions, build the FP64 propagator tables and the
// FFT twiddle tables on the device, and pick the team (number of CTAs that
// share one field).  Propagation of a single field is one cooperative
// persistent launch: the team loops over all slices, its CTAs handing the
// field to each other twice per slice through tagged elements (see
// bpm_kernels.cuh); grids without a persistent kernel
// run one launch per half-step.  The kernels themselves are compiled in the
// ops_*.cu units and found through the registry of bpm_ops.h.  Every entry
// point returns a status code and records a message for bpm_last_error().
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "bpm.h"
#include "bpm_aux_kernels.cuh"
#include "bpm_ops.h"

using namespace bpmk;

namespace bpmk {

static OpsRegistry& registry() {
  static OpsRegistry r;
  static std::once_flag once;
  std::call_once(once, [] {
    register_ops_small(r);
    register_ops_256(r);
    register_ops_384(r);
    register_ops_512(r);
    register_ops_1024(r);
    register_ops_2048(r);
  });
  return r;
}

const LenOps* find_len_ops(int n, int sched) {
  for (const LenOps& o : registry().lens)
    if (o.n == n && o.sched == sched) return &o;
  return nullptr;
}

const PairOps* find_pair_ops(int nx, int ny, int sched) {
  for (const PairOps& o : registry().pairs)
    if (o.nx == nx && o.ny == ny && o.sched == sched) return &o;
  return nullptr;
}

const std::vector<int>& supported_lengths() {
  static std::vector<int> v = [] {
    std::vector<int> r;
    for (const LenOps& o : registry().lens)
      if (std::find(r.begin(), r.end(), o.n) == r.end()) r.push_back(o.n);
    std::sort(r.begin(), r.end());
    return r;
  }();
  return v;
}

}  // namespace bpmk

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define BPM_CU(call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(BPM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

constexpr double kTwoPi = 6.283185307179586;
constexpr long long kMaxPixels = 1ll << 22;   // nx ny at most (a 2048 x 2048 slice)

bool supported_len(int n) {
  const std::vector<int>& v = supported_lengths();
  return std::find(v.begin(), v.end(), n) != v.end();
}

int default_schedule(int n) {
  for (int s = 0;; ++s) {
    const LenOps* o = find_len_ops(n, s);
    if (!o) return 0;
    if (o->is_default) return s;
  }
}

int schedule_count(int n) {
  const LenOps* o = find_len_ops(n, 0);
  return o ? o->schedules : 0;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// One transform length (and schedule) used by a plan: its kernels and its
// twiddle table on the device.
struct LenRes {
  const LenOps* ops = nullptr;
  float2* tw = nullptr;
};

// The persistent launch of a single-field plan (ops == nullptr: the grid has
// no persistent kernel and runs one launch per half-step).
struct GridRes {
  const PairOps* ops = nullptr;
  float2* tw = nullptr;           // combined row + column table (owned)
  int team = 0;                   // CTAs per field
  size_t smem_persist = 0;        // dynamic shared memory with the staging buffers
  int rmax_r = 0, rmax_c = 0;     // rows / columns per team CTA at most
  int h_res = 0, dn_stage = 0;
};

struct InstPlan {
  bpm_instance_desc d;
  float2* ht = nullptr;
  float* gt = nullptr;      // BPM_FLAG_ADAPTIVE: k0^2 n0 dz / kz0, laid out like ht
  float* delta = nullptr;   // BPM_FLAG_ADAPTIVE: mean index step per slice [nz]
};

struct bpm_plan_s {
  std::vector<InstPlan> inst;
  std::map<std::pair<int, int>, LenRes> lens;   // (length, schedule) -> kernels and table
  std::map<std::pair<int, int>, float2*> tmp;   // (nx, ny) -> field scratch of the input synthesis
  GridRes grid;                     // single-field plans
  int sched = 0;                    // schedule of a single-field square plan
  unsigned flags = 0;
  int dev = 0, sms = 0;
  size_t max_optin = 0;
  unsigned* bar = nullptr;
  int* err = nullptr;
  unsigned long long* npupil = nullptr;
  int* foci_idx = nullptr;
  int* demux_foci = nullptr;        // bpm_demultiplex: device copy of the focus list
  int demux_cap = 0;
  double* foci_phase = nullptr;
  int foci_cap = 0;
  unsigned long long timeout_ns = 2000000000ull;
  unsigned bar_extra = 0;
  int tag_stall = 0;                // test hook (bpm_debug_stall_exchange)
  cudaStream_t last = 0;
  // batched plans (n_inst > 1): one persistent cluster launch
  InstArgs* d_inst = nullptr;
  InstArgs* h_inst = nullptr;       // pinned staging of the per-call instance arguments
  int* d_order = nullptr;
  std::vector<int> order_h;        // host copy of the queue order
  unsigned long long* d_queue = nullptr;
  int* d_slots = nullptr;
  cudaStream_t fill_stream = nullptr;         // fill launch of small teams (created with the batch setup)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  size_t batch_smem = 0;
  int cluster = 8;                  // CTAs per team (cluster size), set by bpm_autotune
  int batch_set = 0;                // transform schedule set of the batched kernel, set by bpm_autotune
  BatchKernel bk;                   // the batched kernel of that set
  bool have_args = false;           // h_inst holds the arguments of the last call
  cudaStream_t cap = nullptr;       // capture stream for BPM_FLAG_GRAPH
  cudaGraphExec_t gexec = nullptr;
  // host-buffer streaming (bpm_propagate_host): two-slot rings of index and
  // intensity chunks, the field, copy streams and events (created on first use)
  int host_chunk = 0;
  __half* ring_dn[2] = {nullptr, nullptr};
  float* ring_i[2] = {nullptr, nullptr};
  float2* host_field = nullptr;
  cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
  cudaEvent_t ev_h2d[2] = {}, ev_prop[2] = {}, ev_d2h[2] = {};
};

namespace {

// schedules of the row and column lengths of instance i (batched plans: the
// schedule set of the batched kernel)
int row_sched_of(const bpm_plan_s* p, const bpm_instance_desc& d) {
  if (p->inst.size() > 1) return p->bk.sched_of(d.nx);
  return d.nx == d.ny ? p->sched : default_schedule(d.nx);
}
int col_sched_of(const bpm_plan_s* p, const bpm_instance_desc& d) {
  if (p->inst.size() > 1) return p->bk.sched_of(d.ny);
  return d.nx == d.ny ? p->sched : default_schedule(d.ny);
}

BatchKernel batch_kernel(int set) {
  switch (set) {
    case 1: return batch_kernel_1();
    case 2: return batch_kernel_2();
    default: return batch_kernel_0();
  }
}

// The plan's resources for length n in schedule s: kernels' shared-memory
// limits raised and the twiddle table uploaded (once per plan).
int use_length(bpm_plan_s* p, int n, int s, LenRes** out) {
  auto key = std::make_pair(n, s);
  auto it = p->lens.find(key);
  if (it != p->lens.end()) {
    *out = &it->second;
    return BPM_OK;
  }
  const LenOps* o = find_len_ops(n, s);
  if (!o) return fail(BPM_ERR_UNSUPPORTED, "transform length %d has no schedule %d", n, s);
  if (o->smem > p->max_optin || o->line_smem > p->max_optin)
    return fail(BPM_ERR_UNSUPPORTED, "transform length %d needs more shared memory than the device has", n);
  BPM_CU(o->init(o->smem, o->line_smem));
  std::vector<float2> tw;
  o->twiddles(tw);
  if (tw.size() != (size_t)o->tw_count || tw.empty())
    return fail(BPM_ERR_UNSUPPORTED, "twiddle table size mismatch for length %d", n);
  LenRes r;
  r.ops = o;
  BPM_CU(cudaMalloc(&r.tw, tw.size() * sizeof(float2)));
  cudaError_t e = cudaMemcpy(r.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(r.tw);
    return fail(BPM_ERR_CUDA, "twiddle upload failed: %s", cudaGetErrorString(e));
  }
  *out = &(p->lens[key] = r);
  return BPM_OK;
}

// Team and shared-memory staging of the persistent kernel of a grid: the
// smallest team that gives every group one row and one column per half-step
// (every SM takes rows with the four-step column layout), at most one CTA per
// SM; the staging buffers of propagator columns and index rows are dropped
// (in that order) when they would not fit next to the tables and group
// buffers.
void grid_config(const PairOps* o, int nx, int ny, int sms, size_t max_optin, GridRes& g) {
  const int want = o->four_step ? ny : std::max((ny + o->row_ng - 1) / o->row_ng, (nx + o->col_ng - 1) / o->col_ng);
  g.ops = o;
  g.team = std::max(1, std::min(want, sms));
  g.rmax_r = (ny + g.team - 1) / g.team;
  const int cper = (nx + g.team - 1) / g.team;
  g.rmax_c = (cper + o->col_ng - 1) / o->col_ng * o->col_ng;
  auto rup = [](size_t b) { return (b + 15) & ~(size_t)15; };
  const size_t hb = rup((size_t)g.rmax_c * o->col_hs * sizeof(float2)), db = rup((size_t)g.rmax_r * nx * 2);
  const size_t budget = max_optin - 1024;   // static shared memory of the kernel
  const size_t base = o->smem_base;
  g.h_res = g.dn_stage = 1;
  if (base + hb + db > budget) g.h_res = 0;
  if (base + db > budget) g.dn_stage = 0;
  g.smem_persist = base + (g.h_res ? hb : 0) + (g.dn_stage ? db : 0);
}

// The persistent kernel of a single-field plan's grid in its schedule, when
// one is compiled and fits: launch attributes, occupancy check and the
// combined twiddle table.
int setup_grid(bpm_plan_s* p) {
  const bpm_instance_desc& d = p->inst[0].d;
  GridRes& g = p->grid;
  cudaFree(g.tw);
  g = GridRes();
  if (p->flags & BPM_FLAG_MULTI_LAUNCH) return BPM_OK;
  const PairOps* o = find_pair_ops(d.nx, d.ny, d.nx == d.ny ? p->sched : 0);
  if (!o) return BPM_OK;     // one launch per half-step
  GridRes r;
  grid_config(o, d.nx, d.ny, p->sms, p->max_optin, r);
  if (r.smem_persist > p->max_optin - 1024) return BPM_OK;
  for (int k = 0; k < 2; ++k)
    BPM_CU(cudaFuncSetAttribute(o->kernel[k], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r.smem_persist));
  int per_sm = 0;
  BPM_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, o->kernel[0], kThreads, r.smem_persist));
  if (per_sm < 1) return BPM_OK;
  std::vector<float2> tw;
  o->twiddles(tw);
  if (tw.size() != (size_t)o->tw_count || tw.empty())
    return fail(BPM_ERR_UNSUPPORTED, "twiddle table size mismatch for the %d x %d grid", d.nx, d.ny);
  BPM_CU(cudaMalloc(&r.tw, tw.size() * sizeof(float2)));
  cudaError_t e = cudaMemcpy(r.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(r.tw);
    return fail(BPM_ERR_CUDA, "twiddle upload failed: %s", cudaGetErrorString(e));
  }
  g = r;
  return BPM_OK;
}

// Every length, schedule and grid resource of a single-field plan for its
// current schedule.
int setup_single(bpm_plan_s* p) {
  const bpm_instance_desc& d = p->inst[0].d;
  LenRes* lr = nullptr;
  int rc = use_length(p, d.nx, row_sched_of(p, d), &lr);
  if (rc == BPM_OK) rc = use_length(p, d.ny, col_sched_of(p, d), &lr);
  if (rc == BPM_OK) rc = setup_grid(p);
  return rc;
}

int check_desc(const bpm_instance_desc& d, int i) {
  if (!supported_len(d.nx) || !supported_len(d.ny))
    return fail(BPM_ERR_UNSUPPORTED,
                "instance %d: nx = %d or ny = %d is not one of 64, 96, 128, 192, 256, 384, 512, 768, 1024, "
                "1536, 2048", i, d.nx, d.ny);
  if ((long long)d.nx * d.ny > kMaxPixels)
    return fail(BPM_ERR_UNSUPPORTED, "instance %d: nx ny = %lld exceeds 2^22", i, (long long)d.nx * d.ny);
  if (d.nz < 0) return fail(BPM_ERR_ARG, "instance %d: nz < 0", i);
  if (!(d.dx > 0) || !(d.dy > 0) || !(d.dz > 0) || !(d.lambda > 0) || !(d.n0 > 0) || !std::isfinite(d.dx) ||
      !std::isfinite(d.dy) || !std::isfinite(d.dz) || !std::isfinite(d.lambda) || !std::isfinite(d.n0))
    return fail(BPM_ERR_ARG, "instance %d: dx, dy, dz, lambda and n0 must be positive and finite", i);
  return BPM_OK;
}

// lengths the batched kernel is compiled for (square instances only)
bool batch_size_ok(const bpm_instance_desc& d) {
  if (d.nx != d.ny) return false;
  switch (d.nx) {
    case 64: case 128: case 192: case 256: case 384: case 512: case 1024: return true;
    default: return false;
  }
}

// Switch a single-field square plan to schedule sched (the twiddle tables of
// the new schedule, the grid's launch configuration; the propagator tables and
// the synthesis scratch do not depend on it).
int switch_schedule(bpm_plan_s* p, int sched) {
  if (p->sched == sched) return BPM_OK;
  const int keep = p->sched;
  BPM_CU(cudaDeviceSynchronize());      // no launch of this plan may still read the old tables
  p->sched = sched;
  int rc = setup_single(p);
  if (rc) {
    p->sched = keep;
    setup_single(p);
    return rc;
  }
  return BPM_OK;
}

void free_plan(bpm_plan_s* p) {
  if (!p) return;
  for (auto& in : p->inst) {
    cudaFree(in.ht);
    cudaFree(in.gt);
    cudaFree(in.delta);
  }
  for (auto& kv : p->lens) cudaFree(kv.second.tw);
  for (auto& kv : p->tmp) cudaFree(kv.second);
  cudaFree(p->grid.tw);
  cudaFree(p->bar);
  cudaFree(p->err);
  cudaFree(p->npupil);
  cudaFree(p->foci_idx);
  cudaFree(p->demux_foci);
  cudaFree(p->foci_phase);
  cudaFree(p->d_inst);
  cudaFree(p->d_order);
  cudaFree(p->d_queue);
  cudaFree(p->d_slots);
  if (p->h_inst) cudaFreeHost(p->h_inst);
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->fill_stream) cudaStreamDestroy(p->fill_stream);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  for (int k = 0; k < 2; ++k) {
    cudaFree(p->ring_dn[k]);
    cudaFree(p->ring_i[k]);
    if (p->ev_h2d[k]) cudaEventDestroy(p->ev_h2d[k]);
    if (p->ev_prop[k]) cudaEventDestroy(p->ev_prop[k]);
    if (p->ev_d2h[k]) cudaEventDestroy(p->ev_d2h[k]);
  }
  cudaFree(p->host_field);
  if (p->s_h2d) cudaStreamDestroy(p->s_h2d);
  if (p->s_d2h) cudaStreamDestroy(p->s_d2h);
  delete p;
}

StepArgs base_args(bpm_plan_s* p, const InstPlan& in) {
  StepArgs a;
  std::memset(&a, 0, sizeof a);
  a.ht = in.ht;
  a.nx = in.d.nx;
  a.ny = in.d.ny;
  const double k0 = kTwoPi / in.d.lambda;
  a.screen_c = (float)(k0 * in.d.dz);
  a.k0n0 = k0 * in.d.n0;
  a.dx = in.d.dx;
  a.dy = in.d.dy;
  a.bar = p->bar;
  a.err = p->err;
  a.timeout_ns = p->timeout_ns;
  a.bar_extra = p->bar_extra;
  a.tag_stall = p->tag_stall;
  a.carrier = make_float2(1.f, 0.f);
  return a;
}

// ---- launches ---------------------------------------------------------------

// CTAs of a row (column) kernel: one group per row (column) and round at most
// one CTA per SM
int row_grid(const bpm_plan_s* p, const LenOps* o, int rows) {
  return std::max(1, std::min(p->sms, (rows + o->NG - 1) / o->NG));
}

int lens_of(bpm_plan_s* p, const InstPlan& in, const LenRes** rl, const LenRes** cl) {
  auto ir = p->lens.find(std::make_pair(in.d.nx, row_sched_of(p, in.d)));
  auto ic = p->lens.find(std::make_pair(in.d.ny, col_sched_of(p, in.d)));
  if (ir == p->lens.end() || ic == p->lens.end())
    return fail(BPM_ERR_UNSUPPORTED, "grid %d x %d has no kernels in this plan", in.d.nx, in.d.ny);
  *rl = &ir->second;
  *cl = &ic->second;
  return BPM_OK;
}

int launch_propagate(bpm_plan_s* p, const InstPlan& in, StepArgs a, cudaStream_t s) {
  const GridRes& g = p->grid;
  if (!g.ops) {
    // one launch per half-step: rows with the row length's kernels and table,
    // columns with the column length's
    const LenRes *rl, *cl;
    int rc = lens_of(p, in, &rl, &cl);
    if (rc) return rc;
    const int gr = row_grid(p, rl->ops, in.d.ny), gc = row_grid(p, cl->ops, in.d.nx);
    StepArgs ar = a, ac = a;
    ar.tw = rl->tw;
    ac.tw = cl->tw;
    ac.flip_col = rl->ops->loop != cl->ops->loop;
    BPM_CU(rl->ops->row(ROW_FWD, false, gr, ar, a.z_begin, s));
    for (int zi = a.z_begin; zi < a.z_end; ++zi) {
      const int z = a.reverse ? a.z_begin + a.z_end - 1 - zi : zi;     // slice crossed by this step
      BPM_CU(cl->ops->col(COL_PROP, gc, ac, z, s));
      const bool last = zi + 1 == a.z_end;
      BPM_CU(rl->ops->row(last ? ROW_LAST : ROW_STEP, a.kappa != nullptr, gr, ar, z, s));
    }
    return BPM_OK;
  }
  a.tw = g.tw;
  a.rmax_r = g.rmax_r;
  a.rmax_c = g.rmax_c;
  a.h_res = g.h_res;
  a.dn_stage = g.dn_stage;
  BPM_CU(cudaMemsetAsync(p->bar, 0, sizeof(unsigned), s));
  void* args[] = {&a};
  BPM_CU(cudaLaunchCooperativeKernel(g.ops->kernel[a.kappa ? 1 : 0], dim3(g.team), dim3(kThreads), args,
                                     g.smem_persist, s));
  return BPM_OK;
}

// multiplexed synthesis of one focal-depth group: forward 2D DFT of the
// scattered emitters, focusing filter, inverse DFT accumulated into the output
int launch_synth_group(bpm_plan_s* p, const InstPlan& in, StepArgs a, cudaStream_t s) {
  const LenRes *rl, *cl;
  int rc = lens_of(p, in, &rl, &cl);
  if (rc) return rc;
  const int gr = row_grid(p, rl->ops, in.d.ny), gc = row_grid(p, cl->ops, in.d.nx);
  StepArgs ar = a, ac = a;
  ar.tw = rl->tw;
  ac.tw = cl->tw;
  BPM_CU(rl->ops->row(ROW_FWD, false, gr, ar, 0, s));
  BPM_CU(cl->ops->col(COL_FOCUS, gc, ac, 0, s));
  BPM_CU(rl->ops->row(ROW_INV_ACC, false, gr, ar, 0, s));
  return BPM_OK;
}

int launch_light_sheet(bpm_plan_s* p, const InstPlan& in, StepArgs a, double w0, double xc, cudaStream_t s) {
  const LenRes *rl, *cl;
  int rc = lens_of(p, in, &rl, &cl);
  if (rc) return rc;
  a.tw = rl->tw;
  const long long M = (long long)in.d.nx * in.d.ny;
  const int grid = (int)std::max(1ll, std::min<long long>(p->sms, (M + 4 * kThreads - 1) / (4 * kThreads)));
  BPM_CU(rl->ops->light_sheet(grid, a, w0, xc, s));
  return BPM_OK;
}

int finish_call(bpm_plan_s* p, cudaStream_t s) {
  p->last = s;
  if (p->flags & BPM_FLAG_SYNC) return bpm_check(p);
  return BPM_OK;
}

// ---- batched plans -------------------------------------------------------------

// Work estimate of one instance: slices x (transform work of one slice).
double instance_cost(const bpm_instance_desc& d) {
  const double M = (double)d.nx * d.ny;
  return (double)d.nz * M * std::log2(M);
}

int max_active_clusters(bpm_plan_s* p, int cl, int* out) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cl * std::max(1, p->sms / cl));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = p->batch_smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BPM_CU(cudaOccupancyMaxActiveClusters(out, p->bk.fn, &cfg));
  return BPM_OK;
}

// The batched kernel of schedule set `set`: the tables of its schedules for
// the plan's sizes, its shared memory (the largest need of those sizes) and
// launch attributes.
int use_batch_set(bpm_plan_s* p, int set) {
  p->batch_set = set;
  p->bk = batch_kernel(set);
  size_t smem = 0;
  for (const InstPlan& in : p->inst) {
    LenRes* lr = nullptr;
    int rc = use_length(p, in.d.nx, p->bk.sched_of(in.d.nx), &lr);
    if (rc) return rc;
    smem = std::max(smem, lr->ops->smem);
  }
  p->batch_smem = smem;
  BPM_CU(cudaFuncSetAttribute(p->bk.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  BPM_CU(cudaFuncSetAttribute(p->bk.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  return BPM_OK;
}

int setup_batch(bpm_plan_s* p) {
  const int n = (int)p->inst.size();
  int rc0 = use_batch_set(p, 0);
  if (rc0) return rc0;
  BPM_CU(cudaMalloc(&p->d_inst, sizeof(InstArgs) * n));
  BPM_CU(cudaMalloc(&p->d_order, sizeof(int) * n));
  BPM_CU(cudaMalloc(&p->d_queue, sizeof(unsigned long long)));
  BPM_CU(cudaMalloc(&p->d_slots, sizeof(int) * 1024));
  BPM_CU(cudaMallocHost(&p->h_inst, sizeof(InstArgs) * n));
  std::memset(p->h_inst, 0, sizeof(InstArgs) * n);
  // queue order: largest work first (longest-processing-time-first list
  // scheduling over the clusters that pull from the queue)
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return instance_cost(p->inst[a].d) > instance_cost(p->inst[b].d);
  });
  BPM_CU(cudaMemcpy(p->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  p->order_h = order;
  // created here, outside any graph capture of the launches
  BPM_CU(cudaStreamCreateWithFlags(&p->fill_stream, cudaStreamNonBlocking));
  BPM_CU(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
  BPM_CU(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
  int clusters = 0;
  int rc = max_active_clusters(p, p->cluster, &clusters);
  if (rc) return rc;
  if (clusters < 1) return fail(BPM_ERR_UNSUPPORTED, "batched kernel: no cluster of %d CTAs fits", p->cluster);
  return BPM_OK;
}

// Enqueue the batched launch: instance arguments (from pinned host memory),
// queue reset, the cluster launch of the main teams, and a fill launch of
// two-CTA teams on the SMs that whole main clusters leave free (at 8 CTAs per
// cluster 120 of 148 SMs; the fill launch runs on a second stream forked
// after the queue reset and joined back into s, so that both run at once and
// stay inside one captured graph).  The fill teams take instances from the
// small end of the queue, only those small enough not to become the tail.
int enqueue_batch(bpm_plan_s* p, int clusters, cudaStream_t s) {
  const int n = (int)p->inst.size();
  BPM_CU(cudaMemcpyAsync(p->d_inst, p->h_inst, sizeof(InstArgs) * n, cudaMemcpyHostToDevice, s));
  BPM_CU(cudaMemsetAsync(p->d_queue, 0, sizeof(unsigned long long), s));
  // fill teams: positions in the order (largest first) whose cost on a fill
  // team is at most a third of the first one's on a main team, which bounds
  // the tail a fill team can add after the queue runs dry (batch64: 41.2 ms
  // at one half, where the fill teams became the tail; 31.5 ms at a third,
  // 32.0 ms at a quarter, 33.0 ms at a sixth)
  constexpr int kFillCluster = 2, kFillTail = 3;
  const int fill = p->cluster > kFillCluster ? (p->sms - clusters * p->cluster) / kFillCluster : 0;
  int back_min = n;
  if (fill > 0) {
    const double top = instance_cost(p->inst[p->order_h[0]].d);
    while (back_min > 1 &&
           instance_cost(p->inst[p->order_h[back_min - 1]].d) * p->cluster / kFillCluster * kFillTail <= top)
      --back_min;
  }
  const bool use_fill = fill > 0 && back_min < n;
  // the fork follows the argument upload and queue reset, not the main launch
  if (use_fill) BPM_CU(cudaEventRecord(p->ev_fork, s));
  BatchArgs b;
  b.inst = p->d_inst;
  b.order = p->d_order;
  b.n_inst = n;
  b.queue = p->d_queue;
  b.slots = p->d_slots;
  b.slot_base = 0;
  b.from_back = 0;
  b.back_min = 0;
  b.err = p->err;
  b.timeout_ns = p->timeout_ns;
  b.tag_stall = p->tag_stall;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = p->cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(clusters * p->cluster);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = p->batch_smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* kargs[] = {&b};
  BPM_CU(cudaLaunchKernelExC(&cfg, p->bk.fn, kargs));
  if (use_fill) {
    BPM_CU(cudaStreamWaitEvent(p->fill_stream, p->ev_fork, 0));
    BatchArgs f = b;
    f.slot_base = clusters;
    f.from_back = 1;
    f.back_min = back_min;
    attr[0].val.clusterDim.x = kFillCluster;
    cfg.gridDim = dim3(fill * kFillCluster);
    cfg.stream = p->fill_stream;
    void* fargs[] = {&f};
    BPM_CU(cudaLaunchKernelExC(&cfg, p->bk.fn, fargs));
    BPM_CU(cudaEventRecord(p->ev_join, p->fill_stream));
    BPM_CU(cudaStreamWaitEvent(s, p->ev_join, 0));
  }
  return BPM_OK;
}

int propagate_batch(bpm_plan_s* p, const void* const* d_dn, const void* const* d_Ein, void* const* d_Eout,
                    float* const* d_I, int z_begin, int z_end, const int* w_begin, const int* w_end,
                    cudaStream_t stream) {
  const int n = (int)p->inst.size();
  std::vector<InstArgs> args(n);
  std::memset(args.data(), 0, sizeof(InstArgs) * n);
  for (int i = 0; i < n; ++i) {
    const InstPlan& in = p->inst[i];
    const LenRes& r = p->lens[std::make_pair(in.d.nx, p->bk.sched_of(in.d.nx))];
    InstArgs& a = args[i];
    a.work = static_cast<float2*>(d_Eout[i]);
    a.ein = static_cast<const float2*>(d_Ein[i]);
    a.dn = static_cast<const __half*>(d_dn[i]);
    a.inten = d_I ? d_I[i] : nullptr;
    a.ht = in.ht;
    a.tw = r.tw;
    const double k0 = kTwoPi / in.d.lambda;
    a.screen_c = (float)(k0 * in.d.dz);
    a.n = in.d.nx;
    a.z_begin = std::min(z_begin, in.d.nz);
    a.z_end = std::min(z_end, in.d.nz);
    a.iz0 = w_begin ? w_begin[i] : 0;
    a.iz1 = w_end ? w_end[i] : in.d.nz;
    const double ph = std::fmod(k0 * in.d.n0 * in.d.dz * (double)(a.z_end - a.z_begin), kTwoPi);
    a.carrier = make_float2((float)std::cos(ph), (float)std::sin(ph));
  }
  const bool same = p->have_args && std::memcmp(args.data(), p->h_inst, sizeof(InstArgs) * n) == 0;
  if (!same) {
    // the pinned staging may still feed an earlier launch on this stream
    BPM_CU(cudaStreamSynchronize(p->last));
    BPM_CU(cudaStreamSynchronize(stream));
    std::memcpy(p->h_inst, args.data(), sizeof(InstArgs) * n);
    p->have_args = true;
    if (p->gexec) {
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
    }
  }
  int clusters = 0;
  int rc0 = max_active_clusters(p, p->cluster, &clusters);
  if (rc0) return rc0;
  if (clusters < 1) return fail(BPM_ERR_UNSUPPORTED, "batched kernel: no cluster of %d CTAs fits", p->cluster);
  clusters = std::min(clusters, 1024);
  if (!(p->flags & BPM_FLAG_GRAPH)) return enqueue_batch(p, clusters, stream);
  if (!p->gexec) {
    if (!p->cap) BPM_CU(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    BPM_CU(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_batch(p, clusters, p->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->cap, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail(BPM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(BPM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  BPM_CU(cudaGraphLaunch(p->gexec, stream));
  return BPM_OK;
}

}  // namespace

// ---- C ABI -------------------------------------------------------------------

extern "C" int bpm_plan(bpm_plan_t* out, const bpm_instance_desc* inst, int n_inst, unsigned flags,
                        cudaStream_t stream) {
  if (!out) return fail(BPM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!inst || n_inst < 1 || n_inst > 4096) return fail(BPM_ERR_ARG, "n_inst must be in [1, 4096]");
  if (flags & ~(BPM_FLAG_SYNC | BPM_FLAG_MULTI_LAUNCH | BPM_FLAG_GRAPH | BPM_FLAG_ADAPTIVE))
    return fail(BPM_ERR_ARG, "unknown flag bits 0x%x", flags);
  if ((flags & BPM_FLAG_ADAPTIVE) && n_inst > 1)
    return fail(BPM_ERR_UNSUPPORTED, "BPM_FLAG_ADAPTIVE takes single-instance plans");
  for (int i = 0; i < n_inst; ++i) {
    int rc = check_desc(inst[i], i);
    if (rc) return rc;
    if (n_inst > 1 && !batch_size_ok(inst[i]))
      return fail(BPM_ERR_UNSUPPORTED,
                  "instance %d: batched plans take square grids of 64, 128, 192, 256, 384, 512 or 1024 (got %d x %d)",
                  i, inst[i].nx, inst[i].ny);
  }
  bpm_plan_s* p = new (std::nothrow) bpm_plan_s;
  if (!p) return fail(BPM_ERR_ARG, "out of host memory");
  p->flags = flags;
  int rc = BPM_OK;
  auto cu = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == BPM_OK) rc = fail(BPM_ERR_CUDA, "%s failed: %s", what, cudaGetErrorString(e));
    return e == cudaSuccess;
  };
  int optin = 0;
  cu(cudaGetDevice(&p->dev), "cudaGetDevice");
  if (rc == BPM_OK) cu(cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->dev), "cudaDeviceGetAttribute");
  if (rc == BPM_OK)
    cu(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->dev), "cudaDeviceGetAttribute");
  p->max_optin = (size_t)optin;
  if (rc == BPM_OK) cu(cudaMalloc(&p->bar, 64), "cudaMalloc(barrier)");
  if (rc == BPM_OK) cu(cudaMalloc(&p->err, sizeof(int)), "cudaMalloc(error word)");
  if (rc == BPM_OK) cu(cudaMalloc(&p->npupil, sizeof(unsigned long long)), "cudaMalloc(pupil count)");
  if (rc == BPM_OK) cu(cudaMemset(p->err, 0, sizeof(int)), "cudaMemset");
  for (int i = 0; i < n_inst && rc == BPM_OK; ++i) {
    InstPlan ip;
    ip.d = inst[i];
    const size_t M = (size_t)inst[i].nx * inst[i].ny;
    if (!cu(cudaMalloc(&ip.ht, M * sizeof(float2)), "cudaMalloc(propagator)")) break;
    if (flags & BPM_FLAG_ADAPTIVE) {
      if (!cu(cudaMalloc(&ip.gt, M * sizeof(float)), "cudaMalloc(adapted propagator rates)")) {
        cudaFree(ip.ht);
        break;
      }
      if (!cu(cudaMalloc(&ip.delta, std::max(1, inst[i].nz) * sizeof(float)), "cudaMalloc(slice means)")) {
        cudaFree(ip.ht);
        cudaFree(ip.gt);
        break;
      }
    }
    p->inst.push_back(ip);
    const int threads = 256;
    bpm_build_ht_kernel<<<(unsigned)((M + threads - 1) / threads), threads, 0, stream>>>(
        ip.ht, inst[i].nx, inst[i].ny, inst[i].dx, inst[i].dy, inst[i].dz, inst[i].lambda, inst[i].n0);
    cu(cudaGetLastError(), "bpm_build_ht_kernel");
    if (ip.gt) {
      bpm_build_gt_kernel<<<(unsigned)((M + threads - 1) / threads), threads, 0, stream>>>(
          ip.gt, inst[i].nx, inst[i].ny, inst[i].dx, inst[i].dy, inst[i].dz, inst[i].lambda, inst[i].n0);
      cu(cudaGetLastError(), "bpm_build_gt_kernel");
    }
  }
  if (rc == BPM_OK) {
    if (n_inst == 1) {
      const bpm_instance_desc& d = inst[0];
      p->sched = d.nx == d.ny ? default_schedule(d.nx) : 0;
      rc = setup_single(p);
    } else {
      rc = setup_batch(p);
    }
  }
  if (rc == BPM_OK) cu(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
  if (rc != BPM_OK) {
    free_plan(p);
    return rc;
  }
  p->last = stream;
  *out = p;
  return BPM_OK;
}

namespace {

int propagate_impl(bpm_plan_t p, const void* const* d_dn, const void* const* d_Ein, void* const* d_Eout,
                   float* const* d_I, int z_begin, int z_end, const int* w_begin, const int* w_end,
                   cudaStream_t stream, bool reverse = false, const void* d_kappa = nullptr) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  if (!d_dn || !d_Ein || !d_Eout) return fail(BPM_ERR_ARG, "d_dn, d_Ein and d_Eout must be non-NULL arrays");
  if (z_begin < 0 || z_end < z_begin) return fail(BPM_ERR_ARG, "need 0 <= z_begin <= z_end");
  if ((w_begin == nullptr) != (w_end == nullptr)) return fail(BPM_ERR_ARG, "give both window arrays or neither");
  if (w_begin)
    for (size_t i = 0; i < p->inst.size(); ++i)
      if (w_begin[i] < 0 || w_end[i] < w_begin[i])
        return fail(BPM_ERR_ARG, "instance %zu: need 0 <= w_begin <= w_end", i);
  for (size_t i = 0; i < p->inst.size(); ++i) {
    const InstPlan& in = p->inst[i];
    const int zb = std::min(z_begin, in.d.nz), ze = std::min(z_end, in.d.nz);
    if (!d_Ein[i] || !d_Eout[i] || (ze > zb && !d_dn[i]))
      return fail(BPM_ERR_ARG, "instance %zu: NULL device pointer", i);
    if (!aligned16(d_Ein[i]) || !aligned16(d_Eout[i]) || !aligned16(d_dn[i]) || (d_I && !aligned16(d_I[i])))
      return fail(BPM_ERR_ALIGN, "instance %zu: device pointers must be 16-byte aligned", i);
  }
  if (reverse && p->inst.size() > 1) return fail(BPM_ERR_UNSUPPORTED, "reverse propagation takes single-instance plans");
  if (d_kappa && (p->inst.size() > 1 || reverse || (p->flags & BPM_FLAG_ADAPTIVE)))
    return fail(BPM_ERR_UNSUPPORTED, "absorption takes forward propagations of single-instance plans without "
                                     "BPM_FLAG_ADAPTIVE");
  if (d_kappa && !aligned16(d_kappa)) return fail(BPM_ERR_ALIGN, "d_kappa must be 16-byte aligned");
  if (p->inst.size() > 1) {
    int rc = propagate_batch(p, d_dn, d_Ein, d_Eout, d_I, z_begin, z_end, w_begin, w_end, stream);
    if (rc) return rc;
    return finish_call(p, stream);
  }
  for (size_t i = 0; i < p->inst.size(); ++i) {
    const InstPlan& in = p->inst[i];
    const int zb = std::min(z_begin, in.d.nz), ze = std::min(z_end, in.d.nz);
    const size_t bytes = (size_t)in.d.nx * in.d.ny * sizeof(float2);
    if (ze == zb) {
      if (d_Eout[i] != d_Ein[i])
        BPM_CU(cudaMemcpyAsync(d_Eout[i], d_Ein[i], bytes, cudaMemcpyDeviceToDevice, stream));
      continue;
    }
    StepArgs a = base_args(p, in);
    a.work = static_cast<float2*>(d_Eout[i]);
    a.ein = static_cast<const float2*>(d_Ein[i]);
    a.dn = static_cast<const __half*>(d_dn[i]);
    a.inten = d_I ? d_I[i] : nullptr;
    a.iz0 = w_begin ? w_begin[i] : 0;
    a.iz1 = w_end ? w_end[i] : in.d.nz;
    a.z_begin = zb;
    a.z_end = ze;
    a.reverse = reverse ? 1 : 0;
    a.kappa = static_cast<const __half*>(d_kappa);
    if (in.delta) {
      // reading B: mean index step of slices [zb, ze) before the propagation
      // (delta is indexed by absolute slice, as dn is)
      bpm_slice_mean_kernel<<<ze - zb, kThreads, 0, stream>>>(a.dn + (size_t)zb * in.d.nx * in.d.ny,
                                                              (size_t)in.d.nx * in.d.ny, in.delta + zb);
      BPM_CU(cudaGetLastError());
      a.delta = in.delta;
      a.gt = in.gt;
    }
    const double k0 = kTwoPi / in.d.lambda;
    double ph = std::fmod(k0 * in.d.n0 * in.d.dz * (double)(ze - zb), kTwoPi);
    a.carrier = make_float2((float)std::cos(ph), (float)std::sin(ph));
    int rc = launch_propagate(p, in, a, stream);
    if (rc) return rc;
  }
  return finish_call(p, stream);
}

}  // namespace

extern "C" int bpm_propagate(bpm_plan_t p, const void* const* d_dn, const void* const* d_Ein, void* const* d_Eout,
                             float* const* d_I, int z_begin, int z_end, cudaStream_t stream) {
  return propagate_impl(p, d_dn, d_Ein, d_Eout, d_I, z_begin, z_end, nullptr, nullptr, stream);
}

extern "C" int bpm_propagate_window(bpm_plan_t p, const void* const* d_dn, const void* const* d_Ein,
                                    void* const* d_Eout, float* const* d_I, int z_begin, int z_end,
                                    const int* h_w_begin, const int* h_w_end, cudaStream_t stream) {
  if (!h_w_begin || !h_w_end) return fail(BPM_ERR_ARG, "h_w_begin and h_w_end must be non-NULL");
  return propagate_impl(p, d_dn, d_Ein, d_Eout, d_I, z_begin, z_end, h_w_begin, h_w_end, stream);
}

extern "C" int bpm_propagate_reverse(bpm_plan_t p, const void* d_dn, const void* d_Ein, void* d_Eout, float* d_I,
                                     int z_begin, int z_end, cudaStream_t stream) {
  const void* dn[1] = {d_dn};
  const void* ein[1] = {d_Ein};
  void* eout[1] = {d_Eout};
  float* inten[1] = {d_I};
  return propagate_impl(p, dn, ein, eout, d_I ? inten : nullptr, z_begin, z_end, nullptr, nullptr, stream, true);
}

extern "C" int bpm_propagate_absorbing(bpm_plan_t p, const void* d_dn, const void* d_kappa, const void* d_Ein,
                                       void* d_Eout, float* d_I, int z_begin, int z_end, cudaStream_t stream) {
  if (!d_kappa) return fail(BPM_ERR_ARG, "d_kappa is NULL");
  const void* dn[1] = {d_dn};
  const void* ein[1] = {d_Ein};
  void* eout[1] = {d_Eout};
  float* inten[1] = {d_I};
  return propagate_impl(p, dn, ein, eout, d_I ? inten : nullptr, z_begin, z_end, nullptr, nullptr, stream, false,
                        d_kappa);
}

extern "C" int bpm_phase_conjugate(bpm_plan_t p, int inst, void* d_E, cudaStream_t stream) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  if (inst < 0 || inst >= (int)p->inst.size()) return fail(BPM_ERR_ARG, "instance %d out of range", inst);
  if (!d_E) return fail(BPM_ERR_ARG, "d_E is NULL");
  if (!aligned16(d_E)) return fail(BPM_ERR_ALIGN, "d_E must be 16-byte aligned");
  const size_t M = (size_t)p->inst[inst].d.nx * p->inst[inst].d.ny;
  const int grid = (int)std::min<size_t>((M + kThreads - 1) / kThreads, (size_t)p->sms * 8);
  bpm_conj_kernel<<<grid, kThreads, 0, stream>>>(static_cast<float2*>(d_E), M);
  BPM_CU(cudaGetLastError());
  return finish_call(p, stream);
}

extern "C" int bpm_demultiplex(bpm_plan_t p, int inst, const float* d_I, int w_begin, int w_nz, int n_foci,
                               const int* h_foci, int px, int py, int pz, float* d_out, cudaStream_t stream) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  if (inst < 0 || inst >= (int)p->inst.size()) return fail(BPM_ERR_ARG, "instance %d out of range", inst);
  if (w_begin < 0 || w_nz < 0) return fail(BPM_ERR_ARG, "need w_begin >= 0 and w_nz >= 0");
  if (n_foci < 0 || n_foci > (1 << 24)) return fail(BPM_ERR_ARG, "n_foci must be in [0, 2^24]");
  if (px < 1 || py < 1 || pz < 1 || (long long)px * py * pz > (1LL << 30))
    return fail(BPM_ERR_ARG, "patch sizes must be positive and hold at most 2^30 voxels");
  if (n_foci == 0) return finish_call(p, stream);
  if (!h_foci || !d_out || (w_nz > 0 && !d_I)) return fail(BPM_ERR_ARG, "NULL pointer");
  const int nx = p->inst[inst].d.nx, ny = p->inst[inst].d.ny;
  for (int j = 0; j < n_foci; ++j) {
    const int x = h_foci[3 * j], y = h_foci[3 * j + 1];
    if (x < 0 || x >= nx || y < 0 || y >= ny) return fail(BPM_ERR_ARG, "focus %d lies outside the grid", j);
  }
  if ((int)(3 * (size_t)n_foci) > p->demux_cap) {
    BPM_CU(cudaStreamSynchronize(stream));
    cudaFree(p->demux_foci);
    p->demux_foci = nullptr;
    p->demux_cap = 0;
    BPM_CU(cudaMalloc(&p->demux_foci, 3 * (size_t)n_foci * sizeof(int)));
    p->demux_cap = 3 * n_foci;
  }
  // staged through a pageable copy, so the copy completes before the call
  // returns and the caller may reuse h_foci (pinned or not)
  const std::vector<int> foci(h_foci, h_foci + 3 * (size_t)n_foci);
  BPM_CU(cudaMemcpyAsync(p->demux_foci, foci.data(), foci.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
  const long long total = (long long)px * py * pz * n_foci;
  const int grid = (int)std::min<long long>((total + kThreads - 1) / kThreads, (long long)p->sms * 16);
  bpm_demux_kernel<<<grid, kThreads, 0, stream>>>(d_I, nx, ny, w_begin, w_nz, p->demux_foci, n_foci, px, py, pz,
                                                  d_out);
  BPM_CU(cudaGetLastError());
  return finish_call(p, stream);
}

namespace {

int multiplex_impl(bpm_plan_t p, int inst, int n_foci, const double* h_xyz, const double* h_phase, double NA_in,
                   double NA, void* d_Eout, cudaStream_t stream) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  if (inst < 0 || inst >= (int)p->inst.size()) return fail(BPM_ERR_ARG, "instance %d out of range", inst);
  if (n_foci < 0 || n_foci > (1 << 20)) return fail(BPM_ERR_ARG, "n_foci must be in [0, 1048576]");
  if (n_foci > 0 && (!h_xyz || !h_phase)) return fail(BPM_ERR_ARG, "h_xyz and h_phase must be non-NULL");
  if (!(NA > 0) || !std::isfinite(NA)) return fail(BPM_ERR_ARG, "NA must be positive");
  if (!(NA_in >= 0) || !(NA_in < NA)) return fail(BPM_ERR_ARG, "need 0 <= NA_in < NA");
  if (!d_Eout) return fail(BPM_ERR_ARG, "d_Eout is NULL");
  if (!aligned16(d_Eout)) return fail(BPM_ERR_ALIGN, "d_Eout must be 16-byte aligned");
  const InstPlan& in = p->inst[inst];
  const int nx = in.d.nx, ny = in.d.ny;
  const size_t M = (size_t)nx * ny;
  // emitters on the grid, grouped by focal depth (stable order within a group)
  std::vector<int> order;
  for (int j = 0; j < n_foci; ++j) {
    const double x = h_xyz[3 * j], y = h_xyz[3 * j + 1], z = h_xyz[3 * j + 2];
    if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z) || !std::isfinite(h_phase[j]))
      return fail(BPM_ERR_ARG, "emitter %d has a non-finite coordinate or phase", j);
    const double fx = std::floor(x / in.d.dx + 0.5), fy = std::floor(y / in.d.dy + 0.5);
    if (fx < 0 || fx >= nx || fy < 0 || fy >= ny) continue;
    order.push_back(j);
  }
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return h_xyz[3 * a + 2] < h_xyz[3 * b + 2]; });
  if (order.empty()) {
    BPM_CU(cudaMemsetAsync(d_Eout, 0, M * sizeof(float2), stream));
    return finish_call(p, stream);
  }
  if ((int)order.size() > p->foci_cap) {
    BPM_CU(cudaStreamSynchronize(stream));
    cudaFree(p->foci_idx);
    cudaFree(p->foci_phase);
    p->foci_idx = nullptr;
    p->foci_phase = nullptr;
    p->foci_cap = 0;
    BPM_CU(cudaMalloc(&p->foci_idx, order.size() * sizeof(int)));
    BPM_CU(cudaMalloc(&p->foci_phase, order.size() * sizeof(double)));
    p->foci_cap = (int)order.size();
  }
  float2*& tmp = p->tmp[std::make_pair(nx, ny)];
  if (!tmp) BPM_CU(cudaMalloc(&tmp, M * sizeof(float2)));
  std::vector<int> idx;
  std::vector<double> ph, zs;
  for (int j : order) {
    const int fx = (int)std::floor(h_xyz[3 * j] / in.d.dx + 0.5);
    const int fy = (int)std::floor(h_xyz[3 * j + 1] / in.d.dy + 0.5);
    idx.push_back(fy * nx + fx);
    ph.push_back(h_phase[j]);
    zs.push_back(h_xyz[3 * j + 2]);
  }
  // device staging of the emitter lists (pageable source: the copy completes
  // before cudaMemcpyAsync returns, so the host vectors may go out of scope)
  BPM_CU(cudaMemcpyAsync(p->foci_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
  BPM_CU(cudaMemcpyAsync(p->foci_phase, ph.data(), ph.size() * sizeof(double), cudaMemcpyHostToDevice, stream));
  const double k0 = kTwoPi / in.d.lambda;
  const double kna = k0 * NA;
  const double kin = k0 * NA_in;
  StepArgs a = base_args(p, in);
  a.kna2 = kna * kna;
  a.kin2 = kin * kin;
  BPM_CU(cudaMemsetAsync(p->npupil, 0, sizeof(unsigned long long), stream));
  bpm_pupil_count_kernel<<<(unsigned)((M + 255) / 256), 256, 0, stream>>>(nx, ny, in.d.dx, in.d.dy, a.k0n0, a.kin2,
                                                                         a.kna2, p->npupil);
  BPM_CU(cudaGetLastError());
  size_t g0 = 0;
  int group = 0;
  while (g0 < idx.size()) {
    size_t g1 = g0;
    while (g1 < idx.size() && zs[g1] == zs[g0]) ++g1;
    BPM_CU(cudaMemsetAsync(tmp, 0, M * sizeof(float2), stream));
    const int cnt = (int)(g1 - g0);
    bpm_scatter_kernel<<<(cnt + 127) / 128, 128, 0, stream>>>(tmp, nx, ny, p->foci_idx + g0, p->foci_phase + g0,
                                                              cnt, p->npupil);
    BPM_CU(cudaGetLastError());
    a.work = tmp;
    a.ein = tmp;
    a.out = static_cast<float2*>(d_Eout);
    a.zf = zs[g0];
    a.accumulate = group > 0;
    int rc = launch_synth_group(p, in, a, stream);
    if (rc) return rc;
    g0 = g1;
    ++group;
  }
  return finish_call(p, stream);
}

}  // namespace

extern "C" int bpm_multiplex_psf(bpm_plan_t p, int inst, int n_foci, const double* h_xyz, const double* h_phase,
                                 double NA, void* d_Eout, cudaStream_t stream) {
  return multiplex_impl(p, inst, n_foci, h_xyz, h_phase, 0.0, NA, d_Eout, stream);
}

extern "C" int bpm_multiplex_annular(bpm_plan_t p, int inst, int n_foci, const double* h_xyz,
                                     const double* h_phase, double NA_in, double NA_out, void* d_Eout,
                                     cudaStream_t stream) {
  return multiplex_impl(p, inst, n_foci, h_xyz, h_phase, NA_in, NA_out, d_Eout, stream);
}

extern "C" int bpm_light_sheet(bpm_plan_t p, int inst, double NA, double zf, void* d_Eout, cudaStream_t stream) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  if (inst < 0 || inst >= (int)p->inst.size()) return fail(BPM_ERR_ARG, "instance %d out of range", inst);
  if (!(NA > 0) || !std::isfinite(NA) || !std::isfinite(zf)) return fail(BPM_ERR_ARG, "NA must be positive, zf finite");
  if (!d_Eout) return fail(BPM_ERR_ARG, "d_Eout is NULL");
  if (!aligned16(d_Eout)) return fail(BPM_ERR_ALIGN, "d_Eout must be 16-byte aligned");
  const InstPlan& in = p->inst[inst];
  StepArgs a = base_args(p, in);
  a.work = static_cast<float2*>(d_Eout);
  a.zf = zf;
  const double w0 = in.d.lambda / (M_PI * NA);
  const double xc = (double)(in.d.nx / 2) * in.d.dx;
  int rc = launch_light_sheet(p, in, a, w0, xc, stream);
  if (rc) return rc;
  return finish_call(p, stream);
}

extern "C" int bpm_check(bpm_plan_t p) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  BPM_CU(cudaStreamSynchronize(p->last));
  BPM_CU(cudaGetLastError());
  int e = 0;
  BPM_CU(cudaMemcpy(&e, p->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) {
    BPM_CU(cudaMemset(p->err, 0, sizeof(int)));
    if (e == BPM_ERR_TIMEOUT) return fail(BPM_ERR_TIMEOUT, "a device barrier wait ran out of time");
    if (e == BPM_ERR_NAN) return fail(BPM_ERR_NAN, "non-finite value in the refractive-index volume");
    return fail(e, "device error %d", e);
  }
  return BPM_OK;
}

extern "C" int bpm_free(bpm_plan_t p) {
  if (!p) return BPM_OK;
  cudaStreamSynchronize(p->last);
  free_plan(p);
  return BPM_OK;
}

extern "C" const char* bpm_last_error(void) { return g_last_error.c_str(); }

extern "C" int bpm_plan_info(bpm_plan_t p, int* out, int n_out) {
  if (!p || !out || n_out < 0) return fail(BPM_ERR_ARG, "bad arguments");
  const bpm_instance_desc& d = p->inst[0].d;
  const bool persist = p->grid.ops != nullptr;
  const int nz = d.nz;
  int vals[7] = {0, kThreads, 0, persist ? 1 : 0, persist ? 1 : 1 + 2 * nz, p->sched,
                 d.nx == d.ny ? schedule_count(d.nx) : 1};
  if (persist) {
    vals[0] = p->grid.team;
    vals[2] = (int)p->grid.smem_persist;
  } else {
    const LenRes *rl, *cl;
    if (lens_of(p, p->inst[0], &rl, &cl) == BPM_OK) {
      vals[0] = row_grid(p, rl->ops, d.ny);
      vals[2] = (int)std::max(rl->ops->smem, cl->ops->smem);
    }
  }
  if (p->inst.size() > 1) {
    vals[0] = p->cluster;
    vals[2] = (int)p->batch_smem;
    vals[3] = 1;
    vals[4] = 1;
    vals[5] = p->batch_set;
    vals[6] = kBatchKernels;
  }
  for (int i = 0; i < n_out && i < 7; ++i) out[i] = vals[i];
  return BPM_OK;
}

extern "C" int bpm_propagate_host(bpm_plan_t p, const void* h_dn, const void* Ein, int ein_on_device, void* h_Eout,
                                  float* h_I, int chunk, cudaStream_t stream) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  if (p->inst.size() != 1) return fail(BPM_ERR_UNSUPPORTED, "bpm_propagate_host takes single-instance plans");
  if (!h_dn || !Ein || !h_Eout) return fail(BPM_ERR_ARG, "h_dn, Ein and h_Eout must be non-NULL");
  if (chunk < 1) return fail(BPM_ERR_ARG, "chunk must be >= 1");
  if (ein_on_device && !aligned16(Ein)) return fail(BPM_ERR_ALIGN, "device Ein must be 16-byte aligned");
  const InstPlan& in = p->inst[0];
  const int nz = in.d.nz;
  const size_t M = (size_t)in.d.nx * in.d.ny;
  chunk = std::min(chunk, std::max(nz, 1));
  if (chunk > p->host_chunk) {
    BPM_CU(cudaStreamSynchronize(p->last));
    for (int k = 0; k < 2; ++k) {
      cudaFree(p->ring_dn[k]);
      cudaFree(p->ring_i[k]);
      p->ring_dn[k] = nullptr;
      p->ring_i[k] = nullptr;
    }
    p->host_chunk = 0;
    for (int k = 0; k < 2; ++k) {
      BPM_CU(cudaMalloc(&p->ring_dn[k], (size_t)chunk * M * sizeof(__half)));
      BPM_CU(cudaMalloc(&p->ring_i[k], (size_t)chunk * M * sizeof(float)));
    }
    p->host_chunk = chunk;
  }
  if (!p->host_field) BPM_CU(cudaMalloc(&p->host_field, M * sizeof(float2)));
  if (!p->s_h2d) BPM_CU(cudaStreamCreateWithFlags(&p->s_h2d, cudaStreamNonBlocking));
  if (!p->s_d2h) BPM_CU(cudaStreamCreateWithFlags(&p->s_d2h, cudaStreamNonBlocking));
  for (int k = 0; k < 2; ++k) {
    if (!p->ev_h2d[k]) BPM_CU(cudaEventCreateWithFlags(&p->ev_h2d[k], cudaEventDisableTiming));
    if (!p->ev_prop[k]) BPM_CU(cudaEventCreateWithFlags(&p->ev_prop[k], cudaEventDisableTiming));
    if (!p->ev_d2h[k]) BPM_CU(cudaEventCreateWithFlags(&p->ev_d2h[k], cudaEventDisableTiming));
  }
  // the field enters once; chunks then stream through the two ring slots:
  //   copy-in stream : index chunk k -> slot k%2 (after the propagation of chunk k-2 freed it)
  //   stream         : propagation of chunk k (after its index arrived and the
  //                    intensity slot was drained by chunk k-2's copy-out)
  //   copy-out stream: intensity chunk k -> host (after the propagation of chunk k)
  BPM_CU(cudaMemcpyAsync(p->host_field, Ein, M * sizeof(float2),
                         ein_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream));
  const __half* hdn = static_cast<const __half*>(h_dn);
  const int nchunks = (nz + chunk - 1) / chunk;
  for (int k = 0; k < nchunks; ++k) {
    const int slot = k & 1, z0 = k * chunk, c = std::min(chunk, nz - z0);
    if (k >= 2) BPM_CU(cudaStreamWaitEvent(p->s_h2d, p->ev_prop[slot], 0));
    BPM_CU(cudaMemcpyAsync(p->ring_dn[slot], hdn + (size_t)z0 * M, (size_t)c * M * sizeof(__half),
                           cudaMemcpyHostToDevice, p->s_h2d));
    BPM_CU(cudaEventRecord(p->ev_h2d[slot], p->s_h2d));
    BPM_CU(cudaStreamWaitEvent(stream, p->ev_h2d[slot], 0));
    if (k >= 2 && h_I) BPM_CU(cudaStreamWaitEvent(stream, p->ev_d2h[slot], 0));
    const void* dn_arr[1] = {p->ring_dn[slot]};
    const void* ein_arr[1] = {p->host_field};
    void* eout_arr[1] = {p->host_field};
    float* i_arr[1] = {h_I ? p->ring_i[slot] : nullptr};
    const unsigned keep = p->flags;
    p->flags &= ~(unsigned)BPM_FLAG_SYNC;
    int rc = bpm_propagate(p, dn_arr, ein_arr, eout_arr, i_arr, 0, c, stream);
    p->flags = keep;
    if (rc) return rc;
    BPM_CU(cudaEventRecord(p->ev_prop[slot], stream));
    if (h_I) {
      BPM_CU(cudaStreamWaitEvent(p->s_d2h, p->ev_prop[slot], 0));
      BPM_CU(cudaMemcpyAsync(h_I + (size_t)z0 * M, p->ring_i[slot], (size_t)c * M * sizeof(float),
                             cudaMemcpyDeviceToHost, p->s_d2h));
      BPM_CU(cudaEventRecord(p->ev_d2h[slot], p->s_d2h));
    }
  }
  BPM_CU(cudaMemcpyAsync(h_Eout, p->host_field, M * sizeof(float2), cudaMemcpyDeviceToHost, stream));
  BPM_CU(cudaStreamSynchronize(p->s_h2d));
  BPM_CU(cudaStreamSynchronize(p->s_d2h));
  p->last = stream;
  return bpm_check(p);
}

namespace {
// Single-field plans: time the propagation of slices [0, z_probe) with every
// transform schedule of the plan's size (one warm-up, one timed call each)
// and keep the fastest.
int autotune_schedule(bpm_plan_s* p, const void* const* d_dn, const void* const* d_Ein, void* const* d_Eout,
                      float* const* d_I, int z_probe, cudaStream_t stream) {
  const bpm_instance_desc& d = p->inst[0].d;
  const int count = d.nx == d.ny ? schedule_count(d.nx) : 1;
  if (count < 2) return BPM_OK;
  const int keep = p->sched;
  float best = 1e30f;
  int best_s = keep;
  cudaEvent_t e0, e1;
  BPM_CU(cudaEventCreate(&e0));
  BPM_CU(cudaEventCreate(&e1));
  const int zp = std::min(z_probe, std::max(1, p->inst[0].d.nz));
  for (int sc = 0; sc < count; ++sc) {
    if (switch_schedule(p, sc) != BPM_OK) continue;
    int rc = bpm_propagate(p, d_dn, d_Ein, d_Eout, d_I, 0, zp, stream);   // warm-up
    if (rc == BPM_OK) {
      cudaEventRecord(e0, stream);
      rc = bpm_propagate(p, d_dn, d_Ein, d_Eout, d_I, 0, zp, stream);
      cudaEventRecord(e1, stream);
    }
    if (rc != BPM_OK || cudaEventSynchronize(e1) != cudaSuccess) continue;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_s = sc;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  const int rc = switch_schedule(p, best_s);
  if (rc) return rc;
  return bpm_check(p);
}
}  // namespace

extern "C" int bpm_set_schedule(bpm_plan_t p, int schedule) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  if (p->inst.size() != 1) {
    if (schedule < 0 || schedule >= kBatchKernels)
      return fail(BPM_ERR_ARG, "batched plans have schedule sets 0..%d, not %d", kBatchKernels - 1, schedule);
    if (schedule == p->batch_set) return BPM_OK;
    BPM_CU(cudaDeviceSynchronize());
    p->have_args = false;
    if (p->gexec) {
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
    }
    return use_batch_set(p, schedule);
  }
  const bpm_instance_desc& d = p->inst[0].d;
  const int count = d.nx == d.ny ? schedule_count(d.nx) : 1;
  if (schedule < 0 || schedule >= count)
    return fail(BPM_ERR_ARG, "grid %d x %d has schedules 0..%d, not %d", d.nx, d.ny, count - 1, schedule);
  return switch_schedule(p, schedule);
}

extern "C" int bpm_autotune(bpm_plan_t p, const void* const* d_dn, const void* const* d_Ein, void* const* d_Eout,
                            float* const* d_I, int z_probe, cudaStream_t stream) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  if (z_probe < 1) return fail(BPM_ERR_ARG, "z_probe must be >= 1");
  if (p->inst.size() < 2) return autotune_schedule(p, d_dn, d_Ein, d_Eout, d_I, z_probe, stream);
  // batched plans: every schedule set of the batched kernel with every
  // cluster size, one warm-up and one timed call each
  const int keep_cl = p->cluster, keep_set = p->batch_set;
  const unsigned keep_flags = p->flags;
  p->flags &= ~(unsigned)BPM_FLAG_GRAPH;
  float best = 1e30f;
  int best_cl = keep_cl, best_set = keep_set;
  cudaEvent_t e0, e1;
  BPM_CU(cudaEventCreate(&e0));
  BPM_CU(cudaEventCreate(&e1));
  for (int set = 0; set < kBatchKernels; ++set) {
    if (use_batch_set(p, set) != BPM_OK) continue;
    for (int cl : {2, 4, 8, 16}) {
      int clusters = 0;
      p->cluster = cl;
      if (max_active_clusters(p, cl, &clusters) != BPM_OK || clusters < 1) continue;
      int rc = bpm_propagate(p, d_dn, d_Ein, d_Eout, d_I, 0, z_probe, stream);   // warm-up
      if (rc == BPM_OK) {
        cudaEventRecord(e0, stream);
        rc = bpm_propagate(p, d_dn, d_Ein, d_Eout, d_I, 0, z_probe, stream);
        cudaEventRecord(e1, stream);
      }
      if (rc != BPM_OK || cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_cl = cl;
        best_set = set;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  p->flags = keep_flags;
  p->have_args = false;
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  const int rc = use_batch_set(p, best_set);
  p->cluster = best_cl;
  if (rc) return rc;
  return bpm_check(p);
}

extern "C" int bpm_debug_set_barrier_timeout(bpm_plan_t p, unsigned long long timeout_ns, unsigned extra) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  if (timeout_ns == 0) return fail(BPM_ERR_ARG, "timeout must be positive");
  p->timeout_ns = timeout_ns;
  p->bar_extra = extra;
  return BPM_OK;
}

extern "C" int bpm_debug_stall_exchange(bpm_plan_t p, int on) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  p->tag_stall = on ? 1 : 0;
  return BPM_OK;
}

// ---- allocation-free propagation ----------------------------------------------
//
// For callers that must not allocate device memory (see bpm_propagate_static in
// bpm.h): everything the persistent kernel needs besides the caller's buffers
// lives in one file-scope device array.  Layout: [0, 256) barrier counter
// (offset 0) and error word (offset 64); then the twiddle tables; then the
// transposed propagator table for the largest supported grid.
namespace {

constexpr int kStaticMaxN = 256;
constexpr size_t kStaticWordsBytes = 256;
constexpr size_t kStaticTwiddleFloat2 = 2048;
constexpr size_t kStaticTwiddleBytes = kStaticTwiddleFloat2 * sizeof(float2);
constexpr size_t kStaticPropBytes = (size_t)kStaticMaxN * kStaticMaxN * sizeof(float2);
constexpr size_t kStaticScratchBytes = kStaticWordsBytes + kStaticTwiddleBytes + kStaticPropBytes;

}  // namespace

static __device__ __align__(256) unsigned char bpm_static_scratch[kStaticScratchBytes];

namespace {

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mutex;
unsigned char* g_static_ptr[kStaticMaxDevices] = {};

// Radix schedule of one transform, passed by value to the twiddle kernel;
// `paired` selects the layout the rolled-loop transforms read (LoopFFT: the
// twiddles of r and r + 1 side by side).
struct TwSchedule {
  int n, t, count, sign, paired;
  int r[4];
};

// Same table as append_twiddles(), built on the device in FP64: for pass
// p >= 1 the twiddle W_{Ns R}^{(j mod Ns) r}, j = t + b T, of (b, r, t) goes
// to entry (b R + r) T + t, or with `paired` to ((b R/2 + r/2) T + t) 2 + r%2
// (twiddle_slot(), shared with the host builder).
__global__ void bpm_static_twiddle_kernel(float2* out, TwSchedule s) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (s.count - 1) * s.n) return;
  const int p = 1 + e / s.n, local = e % s.n;
  int Ns = 1;
  for (int i = 0; i < p; ++i) Ns *= s.r[i];
  const int R = s.r[p];
  const int t = local % s.t, br = local / s.t;
  const int r = br % R, b = br / R;
  const int j = t + b * s.t;
  const long long ex = (long long)(j % Ns) * r % (long long)(Ns * R);
  const double ang = s.sign * 6.283185307179586 * (double)ex / (double)(Ns * R);
  double sn, cs;
  sincos(ang, &sn, &cs);
  out[(size_t)(p - 1) * s.n + twiddle_slot(b, r, t, R, s.t, s.paired != 0)] = round_unit(cs, sn);
}

int launch_static_twiddles(const TwSchedule& s, float2* dst, cudaStream_t stream) {
  const int total = (s.count - 1) * s.n;
  if (total <= 0) return BPM_OK;
  bpm_static_twiddle_kernel<<<(total + 255) / 256, 256, 0, stream>>>(dst, s);
  BPM_CU(cudaGetLastError());
  return BPM_OK;
}

int static_propagate(const bpm_instance_desc& d, unsigned char* scratch, const void* d_dn, const void* d_Ein,
                     void* d_Eout, float* d_I, int zb, int ze, cudaStream_t stream) {
  const int N = d.nx;
  const LenOps* lo = find_len_ops(N, 0);
  const PairOps* po = find_pair_ops(N, N, 0);
  if (!lo || !po || lo->four_step || po->tw_count > (int)kStaticTwiddleFloat2)
    return fail(BPM_ERR_UNSUPPORTED, "grid size %d is not supported", N);
  // launch configuration: the same rule as a plan's (grid_config)
  int sms = 0, dev = 0, max_optin = 0;
  BPM_CU(cudaGetDevice(&dev));
  BPM_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BPM_CU(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  GridRes r;
  grid_config(po, N, N, sms, (size_t)max_optin, r);
  BPM_CU(cudaFuncSetAttribute(po->kernel[0], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r.smem_persist));
  unsigned* bar = reinterpret_cast<unsigned*>(scratch);
  int* err = reinterpret_cast<int*>(scratch + 64);
  float2* tw = reinterpret_cast<float2*>(scratch + kStaticWordsBytes);
  float2* ht = reinterpret_cast<float2*>(scratch + kStaticWordsBytes + kStaticTwiddleBytes);
  // the array keeps the previous call's contents: clear the barrier counter
  // and the error word, rebuild both tables
  BPM_CU(cudaMemsetAsync(scratch, 0, kStaticWordsBytes, stream));
  int rc;
  if (lo->loop) {
    TwSchedule s{};
    s.n = N;
    s.t = lo->T;
    s.count = lo->loop_passes;
    s.sign = -1;
    s.paired = 1;
    for (int i = 0; i < lo->loop_passes && i < 4; ++i) s.r[i] = lo->loop_radix;
    rc = launch_static_twiddles(s, tw, stream);
  } else {
    TwSchedule f{}, v{};
    f.n = v.n = N;
    f.t = v.t = lo->T;
    f.count = lo->nf;
    f.sign = -1;
    v.count = lo->ni;
    v.sign = +1;
    for (int i = 0; i < 4; ++i) {
      f.r[i] = lo->rf[i];
      v.r[i] = lo->ri[i];
    }
    rc = launch_static_twiddles(f, tw, stream);
    if (rc == BPM_OK) rc = launch_static_twiddles(v, tw + (size_t)(lo->nf - 1) * N, stream);
  }
  if (rc) return rc;
  const size_t M = (size_t)N * N;
  bpm_build_ht_kernel<<<(unsigned)((M + 255) / 256), 256, 0, stream>>>(ht, d.nx, d.ny, d.dx, d.dy, d.dz, d.lambda,
                                                                       d.n0);
  BPM_CU(cudaGetLastError());
  StepArgs a;
  std::memset(&a, 0, sizeof a);
  a.ht = ht;
  a.tw = tw;
  a.nx = d.nx;
  a.ny = d.ny;
  const double k0 = kTwoPi / d.lambda;
  a.screen_c = (float)(k0 * d.dz);
  a.k0n0 = k0 * d.n0;
  a.dx = d.dx;
  a.dy = d.dy;
  a.bar = bar;
  a.err = err;
  a.timeout_ns = 2000000000ull;
  a.rmax_r = r.rmax_r;
  a.rmax_c = r.rmax_c;
  a.h_res = r.h_res;
  a.dn_stage = r.dn_stage;
  a.work = static_cast<float2*>(d_Eout);
  a.ein = static_cast<const float2*>(d_Ein);
  a.dn = static_cast<const __half*>(d_dn);
  a.inten = d_I;
  a.iz0 = 0;
  a.iz1 = d.nz;
  a.z_begin = zb;
  a.z_end = ze;
  const double ph = std::fmod(k0 * d.n0 * d.dz * (double)(ze - zb), kTwoPi);
  a.carrier = make_float2((float)std::cos(ph), (float)std::sin(ph));
  void* args[] = {&a};
  BPM_CU(cudaLaunchCooperativeKernel(po->kernel[0], dim3(r.team), dim3(kThreads), args, r.smem_persist, stream));
  BPM_CU(cudaStreamSynchronize(stream));
  int e = 0;
  BPM_CU(cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e == BPM_ERR_TIMEOUT) return fail(BPM_ERR_TIMEOUT, "a device barrier wait ran out of time");
  if (e == BPM_ERR_NAN) return fail(BPM_ERR_NAN, "non-finite value in the refractive-index volume");
  if (e != 0) return fail(e, "device error %d", e);
  return BPM_OK;
}

}  // namespace

extern "C" int bpm_propagate_static(const bpm_instance_desc* inst, const void* d_dn, const void* d_Ein,
                                    void* d_Eout, float* d_I, int z_begin, int z_end, cudaStream_t stream) {
  if (!inst) return fail(BPM_ERR_ARG, "inst is NULL");
  int rc = check_desc(*inst, 0);
  if (rc) return rc;
  if (inst->nx != inst->ny || inst->nx > kStaticMaxN)
    return fail(BPM_ERR_UNSUPPORTED,
                "bpm_propagate_static handles square grids up to %d x %d (its fixed device scratch is %zu bytes); "
                "got %d x %d, use bpm_plan/bpm_propagate", kStaticMaxN, kStaticMaxN, kStaticScratchBytes,
                inst->nx, inst->ny);
  if (z_begin < 0 || z_end < z_begin) return fail(BPM_ERR_ARG, "need 0 <= z_begin <= z_end");
  const int zb = std::min(z_begin, inst->nz), ze = std::min(z_end, inst->nz);
  if (!d_Ein || !d_Eout || (ze > zb && !d_dn)) return fail(BPM_ERR_ARG, "NULL device pointer");
  if (!aligned16(d_Ein) || !aligned16(d_Eout) || !aligned16(d_dn) || !aligned16(d_I))
    return fail(BPM_ERR_ALIGN, "device pointers must be 16-byte aligned");
  int dev = 0;
  BPM_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) return fail(BPM_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      BPM_CU(cudaGetSymbolAddress(&p, bpm_static_scratch));
      g_static_ptr[dev] = static_cast<unsigned char*>(p);
    }
    scratch = g_static_ptr[dev];
  }
  if (ze == zb) {
    if (d_Eout != d_Ein)
      BPM_CU(cudaMemcpyAsync(d_Eout, d_Ein, (size_t)inst->nx * inst->ny * sizeof(float2), cudaMemcpyDeviceToDevice,
                             stream));
    BPM_CU(cudaStreamSynchronize(stream));
    return BPM_OK;
  }
  return static_propagate(*inst, scratch, d_dn, d_Ein, d_Eout, d_I, zb, ze, stream);
}
