// bpm.cu - host side of libbpm.so: plans, launches and the C ABI of bpm.h.
//
// Plans validate problem descriptions, build the FP64 propagator tables and the
// FFT twiddle tables on the device, and pick the team (number of CTAs that
// share one field).  Propagation is one cooperative persistent launch per
// instance: the team loops over all slices with two device-wide barriers per
// slice (see bpm_kernels.cuh).  Every entry point returns a status code and
// records a message for bpm_last_error().
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
#include <vector>

#include "bpm.h"
#include "bpm_kernels.cuh"

using namespace bpmk;

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

bool supported_n(int n) {
  switch (n) {
    case 64: case 128: case 192: case 256: case 384: case 512: case 1024: return true;
    default: return false;
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Position of the twiddle of butterfly b, radix element r, thread t within
// one pass's table of a transform with T threads: [b][r][t], or with `paired`
// (LoopFFT, even R) [b][r/2][t][r%2] so that a thread reads the twiddles of
// r and r + 1 with one 16-byte load.  Host and device table builders both use
// it, so their layouts cannot drift apart.
__host__ __device__ inline size_t twiddle_slot(int b, int r, int t, int R, int T, bool paired) {
  return paired ? ((size_t)(b * (R / 2) + r / 2) * T + t) * 2 + (r & 1) : (size_t)(b * R + r) * T + t;
}

// Host-built twiddle table of one transform (FP64, rounded once): for every
// pass p >= 1 of the radix list, N entries holding W_{Ns R}^{(j mod Ns) r},
// j = t + b T, with the transform's sign, laid out [b][r][t], or with
// `paired` (LoopFFT, even R) [b][r/2][t][r%2] so that a thread reads the
// twiddles of r and r + 1 with one 16-byte load.
void append_twiddles(std::vector<float2>& out, int N, int T, const std::vector<int>& radices, int sign,
                     bool paired = false) {
  int Ns = 1;
  for (size_t p = 0; p < radices.size(); ++p) {
    const int R = radices[p];
    if (p > 0) {
      const int B = N / (R * T);
      const size_t base = out.size();
      out.resize(base + (size_t)N);
      for (int b = 0; b < B; ++b)
        for (int r = 0; r < R; ++r)
          for (int t = 0; t < T; ++t) {
            const int j = t + b * T;
            const long long e = (long long)(j % Ns) * r % (long long)(Ns * R);
            const double ang = sign * kTwoPi * (double)e / (double)(Ns * R);
            out[base + twiddle_slot(b, r, t, R, T, paired)] = make_float2((float)std::cos(ang), (float)std::sin(ang));
          }
    }
    Ns *= R;
  }
}

template <class RS>
std::vector<int> radix_list() {
  std::vector<int> r;
  for (int i = 0; i < RS::count; ++i) r.push_back(RS::at(i));
  return r;
}

template <int N, int S = 0>
std::vector<float2> twiddles_for() {
  using C = Cfg<N, S>;
  std::vector<float2> v;
  if constexpr (C::kLoop) {
    append_twiddles(v, N, C::T, std::vector<int>(C::E::NP, C::E::R), -1, true);
  } else {
    append_twiddles(v, N, C::T, radix_list<typename C::F::Rad>(), -1);
    append_twiddles(v, N, C::T, radix_list<typename C::I::Rad>(), +1);
  }
  if constexpr (C::TW4 > 0) {
    // four-step column transform: W_N^(a k), forward sign, laid out
    // [k/2][a][k%2] (the twiddles of k and k + 1 in one 16-byte load)
    const int N1 = C::FS_N1;
    for (int kp = 0; kp < N1 / 2; ++kp)
      for (int a = 0; a < N1; ++a)
        for (int k = 2 * kp; k < 2 * kp + 2; ++k) {
          const long long e = (long long)a * k % N;
          const double ang = -kTwoPi * (double)e / (double)N;
          v.push_back(make_float2((float)std::cos(ang), (float)std::sin(ang)));
        }
  }
  return v;
}

}  // namespace

struct NRes {
  int n = 0;
  float2* tw = nullptr;
  float2* tmp = nullptr;    // N x N scratch for input synthesis (allocated on first use)
  int sched = 0;            // transform schedule (Cfg<n, sched>)
  int team = 0;             // CTAs per field
  size_t smem = 0;          // dynamic shared memory of the half-step kernels
  size_t smem_persist = 0;  // ... of the persistent kernel (with its staging buffers)
  int rmax = 0;             // rows (= columns) per team CTA at most
  int h_res = 0, dn_stage = 0, i_stage = 0;
};

struct InstPlan {
  bpm_instance_desc d;
  float2* ht = nullptr;
  float* gt = nullptr;      // BPM_FLAG_ADAPTIVE: k0^2 n0 dz / kz0, laid out like ht
  float* delta = nullptr;   // BPM_FLAG_ADAPTIVE: mean index step per slice [nz]
};

struct bpm_plan_s {
  std::vector<InstPlan> inst;
  std::map<int, NRes> res;
  unsigned flags = 0;
  int dev = 0, sms = 0;
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

template <int N, int S>
int setup_kernels(NRes& r, int sms) {
  using C = Cfg<N, S>;
  r.smem = cfg_smem_bytes<C>();
  const int smem = (int)r.smem;
  BPM_CU(cudaFuncSetAttribute(bpm_row_kernel<N, ROW_FWD, false, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  BPM_CU(cudaFuncSetAttribute(bpm_row_kernel<N, ROW_STEP, false, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  BPM_CU(cudaFuncSetAttribute(bpm_row_kernel<N, ROW_LAST, false, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  BPM_CU(cudaFuncSetAttribute(bpm_row_kernel<N, ROW_STEP, true, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  BPM_CU(cudaFuncSetAttribute(bpm_row_kernel<N, ROW_LAST, true, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  BPM_CU(cudaFuncSetAttribute(bpm_row_kernel<N, ROW_INV_ACC, false, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  BPM_CU(cudaFuncSetAttribute(bpm_col_kernel<N, COL_PROP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  BPM_CU(cudaFuncSetAttribute(bpm_col_kernel<N, COL_FOCUS, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  BPM_CU(cudaFuncSetAttribute(bpm_light_sheet_kernel<N, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem + (int)(C::GS * sizeof(float2))));
  // smallest team that gives every group one row per half-step, at most one
  // CTA per SM; with the four-step column layout every SM takes rows (fewer
  // rows per CTA) while the columns stay in aligned groups of NG
  const int want = C::FS_N1 > 0 ? N : (N + C::NG - 1) / C::NG;
  r.team = std::max(1, std::min(want, sms));
  // staging buffers of the persistent kernel, dropped (propagator columns
  // first) if they would not fit next to the group buffers
  int max_optin = 0;
  BPM_CU(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, 0));
  // rows (and columns) per CTA at most: columns come in whole groups of NG
  r.rmax = (N + r.team - 1) / r.team;
  r.rmax = (r.rmax + C::NG - 1) / C::NG * C::NG;
  auto rup = [](size_t b) { return (b + 15) & ~(size_t)15; };
  const size_t hb = rup((size_t)r.rmax * C::HS * sizeof(float2)), db = rup((size_t)r.rmax * N * 2),
               ib = rup((size_t)r.rmax * N * sizeof(float));
  const size_t budget = (size_t)max_optin - 1024;   // static shared memory of the kernel
  r.h_res = r.dn_stage = r.i_stage = 1;
  if (r.smem + hb + db + ib > budget) r.h_res = 0;
  if (r.smem + db + ib > budget) r.i_stage = 0;
  if (r.smem + db > budget) r.dn_stage = 0;
  r.smem_persist = r.smem + (r.h_res ? hb : 0) + (r.dn_stage ? db : 0) + (r.i_stage ? ib : 0);
  BPM_CU(cudaFuncSetAttribute(bpm_persistent_kernel<N, false, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)r.smem_persist));
  BPM_CU(cudaFuncSetAttribute((bpm_persistent_kernel<N, true, S>), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)r.smem_persist));
  int per_sm = 0;
  BPM_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bpm_persistent_kernel<N, false, S>, kThreads,
                                                       r.smem_persist));
  if (per_sm < 1) return fail(BPM_ERR_UNSUPPORTED, "persistent kernel for N=%d does not fit on an SM", N);
  std::vector<float2> tw = twiddles_for<N, S>();
  if (tw.size() != (size_t)cfg_twiddles<C>() || tw.empty())
    return fail(BPM_ERR_UNSUPPORTED, "twiddle table size mismatch for N=%d", N);
  r.sched = S;
  BPM_CU(cudaMalloc(&r.tw, tw.size() * sizeof(float2)));
  BPM_CU(cudaMemcpy(r.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
  return BPM_OK;
}

int setup_n(NRes& r, int n, int sms, int sched = 0) {
  r.n = n;
  if (sched < 0 || sched >= kSchedules(n)) return fail(BPM_ERR_ARG, "size %d has no schedule %d", n, sched);
  switch (n * 4 + sched) {
    case 64 * 4: return setup_kernels<64, 0>(r, sms);
    case 128 * 4: return setup_kernels<128, 0>(r, sms);
    case 192 * 4: return setup_kernels<192, 0>(r, sms);
    case 256 * 4: return setup_kernels<256, 0>(r, sms);
    case 256 * 4 + 1: return setup_kernels<256, 1>(r, sms);
    case 256 * 4 + 2: return setup_kernels<256, 2>(r, sms);
    case 384 * 4: return setup_kernels<384, 0>(r, sms);
    case 512 * 4: return setup_kernels<512, 0>(r, sms);
    case 512 * 4 + 1: return setup_kernels<512, 1>(r, sms);
    case 512 * 4 + 2: return setup_kernels<512, 2>(r, sms);
    case 1024 * 4: return setup_kernels<1024, 0>(r, sms);
    case 1024 * 4 + 1: return setup_kernels<1024, 1>(r, sms);
  }
  return fail(BPM_ERR_UNSUPPORTED, "grid size %d is not supported", n);
}

int check_desc(const bpm_instance_desc& d, int i) {
  if (d.nx != d.ny)
    return fail(BPM_ERR_UNSUPPORTED, "instance %d: nx (%d) != ny (%d) is not supported", i, d.nx, d.ny);
  if (!supported_n(d.nx))
    return fail(BPM_ERR_UNSUPPORTED, "instance %d: nx = %d is not one of 64,128,192,256,384,512,1024", i, d.nx);
  if (d.nz < 0) return fail(BPM_ERR_ARG, "instance %d: nz < 0", i);
  if (!(d.dx > 0) || !(d.dy > 0) || !(d.dz > 0) || !(d.lambda > 0) || !(d.n0 > 0) || !std::isfinite(d.dx) ||
      !std::isfinite(d.dy) || !std::isfinite(d.dz) || !std::isfinite(d.lambda) || !std::isfinite(d.n0))
    return fail(BPM_ERR_ARG, "instance %d: dx, dy, dz, lambda and n0 must be positive and finite", i);
  return BPM_OK;
}

// Rebuild the per-size resources of a single-field plan for schedule sched
// (twiddle table and launch configuration; the propagator tables and the
// synthesis scratch do not depend on it).
int switch_schedule(bpm_plan_s* p, int sched) {
  NRes& cur = p->res.begin()->second;
  if (cur.sched == sched) return BPM_OK;
  NRes r;
  int rc = setup_n(r, cur.n, p->sms, sched);
  if (rc) {
    cudaFree(r.tw);
    return rc;
  }
  BPM_CU(cudaDeviceSynchronize());      // no launch of this plan may still read the old table
  cudaFree(cur.tw);
  r.tmp = cur.tmp;
  cur = r;
  return BPM_OK;
}

void free_plan(bpm_plan_s* p) {
  if (!p) return;
  for (auto& in : p->inst) {
    cudaFree(in.ht);
    cudaFree(in.gt);
    cudaFree(in.delta);
  }
  for (auto& kv : p->res) {
    cudaFree(kv.second.tw);
    cudaFree(kv.second.tmp);
  }
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

StepArgs base_args(bpm_plan_s* p, const InstPlan& in, const NRes& r) {
  StepArgs a;
  std::memset(&a, 0, sizeof a);
  a.ht = in.ht;
  a.tw = r.tw;
  const double k0 = kTwoPi / in.d.lambda;
  a.screen_c = (float)(k0 * in.d.dz);
  a.k0n0 = k0 * in.d.n0;
  a.dx = in.d.dx;
  a.dy = in.d.dy;
  a.bar = p->bar;
  a.err = p->err;
  a.timeout_ns = p->timeout_ns;
  a.bar_extra = p->bar_extra;
  a.carrier = make_float2(1.f, 0.f);
  a.rmax = r.rmax;
  a.h_res = r.h_res;
  a.dn_stage = r.dn_stage;
  a.i_stage = r.i_stage;
  return a;
}

// ---- launches ---------------------------------------------------------------

template <int N, int S>
int launch_propagate(bpm_plan_s* p, const NRes& r, StepArgs a, cudaStream_t s) {
  const int G = r.team;
  if (p->flags & BPM_FLAG_MULTI_LAUNCH) {
    bpm_row_kernel<N, ROW_FWD, false, S><<<G, kThreads, r.smem, s>>>(a, a.z_begin);
    for (int zi = a.z_begin; zi < a.z_end; ++zi) {
      const int z = a.reverse ? a.z_begin + a.z_end - 1 - zi : zi;     // slice crossed by this step
      bpm_col_kernel<N, COL_PROP, S><<<G, kThreads, r.smem, s>>>(a, z);
      const bool last = zi + 1 == a.z_end;
      if (a.kappa) {
        if (!last) bpm_row_kernel<N, ROW_STEP, true, S><<<G, kThreads, r.smem, s>>>(a, z);
        else bpm_row_kernel<N, ROW_LAST, true, S><<<G, kThreads, r.smem, s>>>(a, z);
      } else {
        if (!last) bpm_row_kernel<N, ROW_STEP, false, S><<<G, kThreads, r.smem, s>>>(a, z);
        else bpm_row_kernel<N, ROW_LAST, false, S><<<G, kThreads, r.smem, s>>>(a, z);
      }
    }
    BPM_CU(cudaGetLastError());
    return BPM_OK;
  }
  BPM_CU(cudaMemsetAsync(p->bar, 0, sizeof(unsigned), s));
  void* args[] = {&a};
  const void* fn = a.kappa ? (const void*)bpm_persistent_kernel<N, true, S> : (const void*)bpm_persistent_kernel<N, false, S>;
  BPM_CU(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kThreads), args, r.smem_persist, s));
  return BPM_OK;
}

template <int N, int S>
int launch_synth_group(bpm_plan_s*, const NRes& r, StepArgs a, cudaStream_t s) {
  const int G = r.team;
  bpm_row_kernel<N, ROW_FWD, false, S><<<G, kThreads, r.smem, s>>>(a, 0);
  bpm_col_kernel<N, COL_FOCUS, S><<<G, kThreads, r.smem, s>>>(a, 0);
  bpm_row_kernel<N, ROW_INV_ACC, false, S><<<G, kThreads, r.smem, s>>>(a, 0);
  BPM_CU(cudaGetLastError());
  return BPM_OK;
}

template <int N, int S>
int launch_light_sheet(bpm_plan_s* p, const NRes& r, StepArgs a, double w0, double xc, cudaStream_t s) {
  using C = Cfg<N, S>;
  const int grid = std::max(1, std::min(p->sms, (N * N + 4 * kThreads - 1) / (4 * kThreads)));
  bpm_light_sheet_kernel<N, S><<<grid, kThreads, r.smem + C::GS * sizeof(float2), s>>>(a, w0, xc);
  BPM_CU(cudaGetLastError());
  return BPM_OK;
}

// call with the size N and schedule S of r as compile-time constants
#define BPM_DISPATCH(r, call)                                                 \
  switch ((r).n * 4 + (r).sched) {                                            \
    case 64 * 4: { constexpr int N = 64, S = 0; return call; }                \
    case 128 * 4: { constexpr int N = 128, S = 0; return call; }              \
    case 192 * 4: { constexpr int N = 192, S = 0; return call; }              \
    case 256 * 4: { constexpr int N = 256, S = 0; return call; }              \
    case 256 * 4 + 1: { constexpr int N = 256, S = 1; return call; }          \
    case 256 * 4 + 2: { constexpr int N = 256, S = 2; return call; }          \
    case 384 * 4: { constexpr int N = 384, S = 0; return call; }              \
    case 512 * 4: { constexpr int N = 512, S = 0; return call; }              \
    case 512 * 4 + 1: { constexpr int N = 512, S = 1; return call; }          \
    case 512 * 4 + 2: { constexpr int N = 512, S = 2; return call; }          \
    case 1024 * 4: { constexpr int N = 1024, S = 0; return call; }            \
    case 1024 * 4 + 1: { constexpr int N = 1024, S = 1; return call; }        \
  }                                                                           \
  return fail(BPM_ERR_UNSUPPORTED, "grid size %d (schedule %d) is not supported", (r).n, (r).sched);

int dispatch_propagate(bpm_plan_s* p, const NRes& r, const StepArgs& a, cudaStream_t s) {
  BPM_DISPATCH(r, (launch_propagate<N, S>(p, r, a, s)))
}
int dispatch_synth(bpm_plan_s* p, const NRes& r, const StepArgs& a, cudaStream_t s) {
  BPM_DISPATCH(r, (launch_synth_group<N, S>(p, r, a, s)))
}
int dispatch_light_sheet(bpm_plan_s* p, const NRes& r, const StepArgs& a, double w0, double xc, cudaStream_t s) {
  BPM_DISPATCH(r, (launch_light_sheet<N, S>(p, r, a, w0, xc, s)))
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
  BPM_CU(cudaOccupancyMaxActiveClusters(out, (void*)bpm_batch_kernel, &cfg));
  return BPM_OK;
}

int setup_batch(bpm_plan_s* p) {
  const int n = (int)p->inst.size();
  size_t smem = 0;
  for (auto& kv : p->res) smem = std::max(smem, kv.second.smem);
  p->batch_smem = smem;
  BPM_CU(cudaFuncSetAttribute(bpm_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  BPM_CU(cudaFuncSetAttribute(bpm_batch_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
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
  BPM_CU(cudaLaunchKernelEx(&cfg, bpm_batch_kernel, b));
  if (use_fill) {
    BPM_CU(cudaStreamWaitEvent(p->fill_stream, p->ev_fork, 0));
    BatchArgs f = b;
    f.slot_base = clusters;
    f.from_back = 1;
    f.back_min = back_min;
    attr[0].val.clusterDim.x = kFillCluster;
    cfg.gridDim = dim3(fill * kFillCluster);
    cfg.stream = p->fill_stream;
    BPM_CU(cudaLaunchKernelEx(&cfg, bpm_batch_kernel, f));
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
    const NRes& r = p->res[in.d.nx];
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
  }
  bpm_plan_s* p = new (std::nothrow) bpm_plan_s;
  if (!p) return fail(BPM_ERR_ARG, "out of host memory");
  p->flags = flags;
  int rc = BPM_OK;
  auto cu = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == BPM_OK) rc = fail(BPM_ERR_CUDA, "%s failed: %s", what, cudaGetErrorString(e));
    return e == cudaSuccess;
  };
  cu(cudaGetDevice(&p->dev), "cudaGetDevice");
  if (rc == BPM_OK) cu(cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->dev), "cudaDeviceGetAttribute");
  if (rc == BPM_OK) cu(cudaMalloc(&p->bar, 64), "cudaMalloc(barrier)");
  if (rc == BPM_OK) cu(cudaMalloc(&p->err, sizeof(int)), "cudaMalloc(error word)");
  if (rc == BPM_OK) cu(cudaMalloc(&p->npupil, sizeof(unsigned long long)), "cudaMalloc(pupil count)");
  if (rc == BPM_OK) cu(cudaMemset(p->err, 0, sizeof(int)), "cudaMemset");
  for (int i = 0; i < n_inst && rc == BPM_OK; ++i) {
    InstPlan ip;
    ip.d = inst[i];
    const int n = inst[i].nx;
    if (!p->res.count(n)) {
      NRes r;
      rc = setup_n(r, n, p->sms, n_inst == 1 ? kDefaultSchedule(n) : 0);
      p->res[n] = r;
      if (rc) break;
    }
    const size_t M = (size_t)n * n;
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
  if (rc == BPM_OK && n_inst > 1) rc = setup_batch(p);
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
    const NRes& r = p->res[in.d.nx];
    const int zb = std::min(z_begin, in.d.nz), ze = std::min(z_end, in.d.nz);
    const size_t bytes = (size_t)in.d.nx * in.d.ny * sizeof(float2);
    if (ze == zb) {
      if (d_Eout[i] != d_Ein[i])
        BPM_CU(cudaMemcpyAsync(d_Eout[i], d_Ein[i], bytes, cudaMemcpyDeviceToDevice, stream));
      continue;
    }
    StepArgs a = base_args(p, in, r);
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
    int rc = dispatch_propagate(p, r, a, stream);
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
  const int n = p->inst[inst].d.nx;
  for (int j = 0; j < n_foci; ++j) {
    const int x = h_foci[3 * j], y = h_foci[3 * j + 1];
    if (x < 0 || x >= n || y < 0 || y >= n) return fail(BPM_ERR_ARG, "focus %d lies outside the grid", j);
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
  bpm_demux_kernel<<<grid, kThreads, 0, stream>>>(d_I, n, w_begin, w_nz, p->demux_foci, n_foci, px, py, pz, d_out);
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
  NRes& r = p->res[in.d.nx];
  const int n = in.d.nx;
  const size_t M = (size_t)n * n;
  // emitters on the grid, grouped by focal depth (stable order within a group)
  std::vector<int> order;
  for (int j = 0; j < n_foci; ++j) {
    const double x = h_xyz[3 * j], y = h_xyz[3 * j + 1], z = h_xyz[3 * j + 2];
    if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z) || !std::isfinite(h_phase[j]))
      return fail(BPM_ERR_ARG, "emitter %d has a non-finite coordinate or phase", j);
    const double fx = std::floor(x / in.d.dx + 0.5), fy = std::floor(y / in.d.dy + 0.5);
    if (fx < 0 || fx >= n || fy < 0 || fy >= n) continue;
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
  if (!r.tmp) BPM_CU(cudaMalloc(&r.tmp, M * sizeof(float2)));
  std::vector<int> idx;
  std::vector<double> ph, zs;
  for (int j : order) {
    const int fx = (int)std::floor(h_xyz[3 * j] / in.d.dx + 0.5);
    const int fy = (int)std::floor(h_xyz[3 * j + 1] / in.d.dy + 0.5);
    idx.push_back(fy * n + fx);
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
  StepArgs a = base_args(p, in, r);
  a.kna2 = kna * kna;
  a.kin2 = kin * kin;
  BPM_CU(cudaMemsetAsync(p->npupil, 0, sizeof(unsigned long long), stream));
  bpm_pupil_count_kernel<<<(unsigned)((M + 255) / 256), 256, 0, stream>>>(n, in.d.dx, in.d.dy, a.k0n0, a.kin2,
                                                                         a.kna2, p->npupil);
  BPM_CU(cudaGetLastError());
  size_t g0 = 0;
  int group = 0;
  while (g0 < idx.size()) {
    size_t g1 = g0;
    while (g1 < idx.size() && zs[g1] == zs[g0]) ++g1;
    BPM_CU(cudaMemsetAsync(r.tmp, 0, M * sizeof(float2), stream));
    const int cnt = (int)(g1 - g0);
    bpm_scatter_kernel<<<(cnt + 127) / 128, 128, 0, stream>>>(r.tmp, n, p->foci_idx + g0, p->foci_phase + g0, cnt,
                                                              p->npupil);
    BPM_CU(cudaGetLastError());
    a.work = r.tmp;
    a.ein = r.tmp;
    a.out = static_cast<float2*>(d_Eout);
    a.zf = zs[g0];
    a.accumulate = group > 0;
    int rc = dispatch_synth(p, r, a, stream);
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
  const NRes& r = p->res[in.d.nx];
  StepArgs a = base_args(p, in, r);
  a.work = static_cast<float2*>(d_Eout);
  a.zf = zf;
  const double w0 = in.d.lambda / (M_PI * NA);
  const double xc = (double)(in.d.nx / 2) * in.d.dx;
  int rc = dispatch_light_sheet(p, r, a, w0, xc, stream);
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
  const NRes& r = p->res.begin()->second;
  const bool multi = (p->flags & BPM_FLAG_MULTI_LAUNCH) != 0;
  const int nz = p->inst[0].d.nz;
  int vals[7] = {r.team, kThreads, (int)(multi ? r.smem : r.smem_persist), multi ? 0 : 1, multi ? 1 + 2 * nz : 1,
                 r.sched, kSchedules(r.n)};
  if (p->inst.size() > 1) {
    vals[0] = p->cluster;
    vals[2] = (int)p->batch_smem;
    vals[3] = 1;
    vals[4] = 1;
    vals[5] = 0;
    vals[6] = 1;
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
  const int n = p->inst[0].d.nx, count = kSchedules(n);
  if (count < 2) return BPM_OK;
  const int keep = p->res.begin()->second.sched;
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
  if (p->inst.size() != 1) return fail(BPM_ERR_UNSUPPORTED, "schedules are chosen for single-field plans only");
  const int n = p->inst[0].d.nx;
  if (schedule < 0 || schedule >= kSchedules(n))
    return fail(BPM_ERR_ARG, "size %d has schedules 0..%d, not %d", n, kSchedules(n) - 1, schedule);
  return switch_schedule(p, schedule);
}

extern "C" int bpm_autotune(bpm_plan_t p, const void* const* d_dn, const void* const* d_Ein, void* const* d_Eout,
                            float* const* d_I, int z_probe, cudaStream_t stream) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  if (z_probe < 1) return fail(BPM_ERR_ARG, "z_probe must be >= 1");
  if (p->inst.size() < 2) return autotune_schedule(p, d_dn, d_Ein, d_Eout, d_I, z_probe, stream);
  const int keep = p->cluster;
  const unsigned keep_flags = p->flags;
  p->flags &= ~(unsigned)BPM_FLAG_GRAPH;
  float best = 1e30f;
  int best_cl = keep;
  cudaEvent_t e0, e1;
  BPM_CU(cudaEventCreate(&e0));
  BPM_CU(cudaEventCreate(&e1));
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
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  p->cluster = best_cl;
  p->flags = keep_flags;
  p->have_args = false;
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  return bpm_check(p);
}

extern "C" int bpm_debug_set_barrier_timeout(bpm_plan_t p, unsigned long long timeout_ns, unsigned extra) {
  if (!p) return fail(BPM_ERR_ARG, "plan is NULL");
  if (timeout_ns == 0) return fail(BPM_ERR_ARG, "timeout must be positive");
  p->timeout_ns = timeout_ns;
  p->bar_extra = extra;
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
  out[(size_t)(p - 1) * s.n + twiddle_slot(b, r, t, R, s.t, s.paired != 0)] = make_float2((float)cs, (float)sn);
}

template <class RS>
TwSchedule schedule_of(int n, int t, int sign) {
  TwSchedule s{};
  s.n = n;
  s.t = t;
  s.count = RS::count;
  s.sign = sign;
  for (int i = 0; i < RS::count && i < 4; ++i) s.r[i] = RS::at(i);
  return s;
}

int launch_static_twiddles(const TwSchedule& s, float2* dst, cudaStream_t stream) {
  const int total = (s.count - 1) * s.n;
  if (total <= 0) return BPM_OK;
  bpm_static_twiddle_kernel<<<(total + 255) / 256, 256, 0, stream>>>(dst, s);
  BPM_CU(cudaGetLastError());
  return BPM_OK;
}

template <int N>
int static_propagate(const bpm_instance_desc& d, unsigned char* scratch, const void* d_dn, const void* d_Ein,
                     void* d_Eout, float* d_I, int zb, int ze, cudaStream_t stream) {
  using C = Cfg<N>;
  static_assert(cfg_twiddles<C>() <= (int)kStaticTwiddleFloat2 && C::TW4 == 0, "twiddle region too small");
  // launch configuration: the same rule as a plan's (setup_kernels)
  int sms = 0, dev = 0, max_optin = 0;
  BPM_CU(cudaGetDevice(&dev));
  BPM_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BPM_CU(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  NRes r;
  r.n = N;
  r.smem = cfg_smem_bytes<C>();
  r.team = std::max(1, std::min((N + C::NG - 1) / C::NG, sms));
  r.rmax = (N + r.team - 1) / r.team;
  auto rup = [](size_t b) { return (b + 15) & ~(size_t)15; };
  const size_t hb = rup((size_t)r.rmax * C::HS * sizeof(float2)), db = rup((size_t)r.rmax * N * 2),
               ib = rup((size_t)r.rmax * N * sizeof(float));
  const size_t budget = (size_t)max_optin - 1024;
  r.h_res = r.dn_stage = r.i_stage = 1;
  if (r.smem + hb + db + ib > budget) r.h_res = 0;
  if (r.smem + db + ib > budget) r.i_stage = 0;
  if (r.smem + db > budget) r.dn_stage = 0;
  r.smem_persist = r.smem + (r.h_res ? hb : 0) + (r.dn_stage ? db : 0) + (r.i_stage ? ib : 0);
  BPM_CU(cudaFuncSetAttribute(bpm_persistent_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)r.smem_persist));
  unsigned* bar = reinterpret_cast<unsigned*>(scratch);
  int* err = reinterpret_cast<int*>(scratch + 64);
  float2* tw = reinterpret_cast<float2*>(scratch + kStaticWordsBytes);
  float2* ht = reinterpret_cast<float2*>(scratch + kStaticWordsBytes + kStaticTwiddleBytes);
  // the array keeps the previous call's contents: clear the barrier counter
  // and the error word, rebuild both tables
  BPM_CU(cudaMemsetAsync(scratch, 0, kStaticWordsBytes, stream));
  int rc;
  if constexpr (C::kLoop) {
    TwSchedule s{};
    s.n = N;
    s.t = C::T;
    s.count = C::E::NP;
    s.sign = -1;
    s.paired = 1;
    for (int i = 0; i < C::E::NP && i < 4; ++i) s.r[i] = C::E::R;
    rc = launch_static_twiddles(s, tw, stream);
  } else {
    rc = launch_static_twiddles(schedule_of<typename C::F::Rad>(N, C::T, -1), tw, stream);
    if (rc == BPM_OK) rc = launch_static_twiddles(schedule_of<typename C::I::Rad>(N, C::T, +1), tw + C::TWF, stream);
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
  const double k0 = kTwoPi / d.lambda;
  a.screen_c = (float)(k0 * d.dz);
  a.k0n0 = k0 * d.n0;
  a.dx = d.dx;
  a.dy = d.dy;
  a.bar = bar;
  a.err = err;
  a.timeout_ns = 2000000000ull;
  a.rmax = r.rmax;
  a.h_res = r.h_res;
  a.dn_stage = r.dn_stage;
  a.i_stage = r.i_stage;
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
  BPM_CU(cudaLaunchCooperativeKernel((const void*)bpm_persistent_kernel<N>, dim3(r.team), dim3(kThreads), args,
                                     r.smem_persist, stream));
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
  if (inst->nx > kStaticMaxN)
    return fail(BPM_ERR_UNSUPPORTED,
                "bpm_propagate_static handles grids up to %d x %d (its fixed device scratch is %zu bytes); "
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
  switch (inst->nx) {
    case 64: return static_propagate<64>(*inst, scratch, d_dn, d_Ein, d_Eout, d_I, zb, ze, stream);
    case 128: return static_propagate<128>(*inst, scratch, d_dn, d_Ein, d_Eout, d_I, zb, ze, stream);
    case 192: return static_propagate<192>(*inst, scratch, d_dn, d_Ein, d_Eout, d_I, zb, ze, stream);
    case 256: return static_propagate<256>(*inst, scratch, d_dn, d_Ein, d_Eout, d_I, zb, ze, stream);
  }
  return fail(BPM_ERR_UNSUPPORTED, "grid size %d is not supported", inst->nx);
}
