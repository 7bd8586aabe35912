// bpm_ops.cuh - instantiation of the templated kernels for one transform
// length (LenImpl) or one grid (PairImpl), and the records that describe them
// to the host side (bpm_ops.h).  Included by the kernel translation units
// (ops_*.cu) only.
#pragma once
#include <cmath>
#include <vector>

#include "bpm_kernels.cuh"
#include "bpm_ops.h"

namespace bpmk {

constexpr double kTwoPiHost = 6.283185307179586;

// Host-built twiddle table of one transform (FP64, rounded by round_unit): for every
// pass p >= 1 of the radix list, N entries holding W_{Ns R}^{(j mod Ns) r},
// j = t + b T, with the transform's sign, at twiddle_slot(b, r, t).
inline void append_twiddles(std::vector<float2>& out, int N, int T, const std::vector<int>& radices, int sign,
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
            const double ang = sign * kTwoPiHost * (double)e / (double)(Ns * R);
            out[base + twiddle_slot(b, r, t, R, T, paired)] = round_unit(std::cos(ang), std::sin(ang));
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

// The full table of one length's configuration: forward, inverse, four-step.
template <class C>
void cfg_twiddles_host(std::vector<float2>& v) {
  if constexpr (C::kLoop) {
    append_twiddles(v, C::N, C::T, std::vector<int>(C::E::NP, C::E::R), -1, true);
  } else {
    append_twiddles(v, C::N, C::T, radix_list<typename C::F::Rad>(), -1);
    append_twiddles(v, C::N, C::T, radix_list<typename C::I::Rad>(), +1);
  }
  if constexpr (C::TW4 > 0) {
    // four-step column transform: W_N^(a k), forward sign, laid out
    // [k/2][a][k%2] (the twiddles of k and k + 1 in one 16-byte load)
    const int N1 = C::FS_N1, N = C::N;
    for (int kp = 0; kp < N1 / 2; ++kp)
      for (int a = 0; a < N1; ++a)
        for (int k = 2 * kp; k < 2 * kp + 2; ++k) {
          const long long e = (long long)a * k % N;
          const double ang = -kTwoPiHost * (double)e / (double)N;
          v.push_back(round_unit(std::cos(ang), std::sin(ang)));
        }
  }
}

template <class C>
struct LenImpl {
  static constexpr size_t kSmem = cfg_smem_bytes<C>();
  static constexpr size_t kLineSmem = kSmem + C::GS * sizeof(float2);

  static cudaError_t init(size_t smem, size_t line) {
    const int s = (int)smem, l = (int)line;
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* fn, int bytes) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    set((const void*)bpm_row_kernel<C, ROW_FWD, false>, s);
    set((const void*)bpm_row_kernel<C, ROW_STEP, false>, s);
    set((const void*)bpm_row_kernel<C, ROW_LAST, false>, s);
    set((const void*)bpm_row_kernel<C, ROW_STEP, true>, s);
    set((const void*)bpm_row_kernel<C, ROW_LAST, true>, s);
    set((const void*)bpm_row_kernel<C, ROW_INV_ACC, false>, s);
    set((const void*)bpm_col_kernel<C, COL_PROP>, s);
    set((const void*)bpm_col_kernel<C, COL_FOCUS>, s);
    set((const void*)bpm_light_sheet_kernel<C>, l);
    return e;
  }

  static cudaError_t row(int mode, bool kappa, int grid, const StepArgs& a, int z, cudaStream_t s) {
    switch (mode * 2 + (kappa ? 1 : 0)) {
      case ROW_FWD * 2: bpm_row_kernel<C, ROW_FWD, false><<<grid, kThreads, kSmem, s>>>(a, z); break;
      case ROW_STEP * 2: bpm_row_kernel<C, ROW_STEP, false><<<grid, kThreads, kSmem, s>>>(a, z); break;
      case ROW_STEP * 2 + 1: bpm_row_kernel<C, ROW_STEP, true><<<grid, kThreads, kSmem, s>>>(a, z); break;
      case ROW_LAST * 2: bpm_row_kernel<C, ROW_LAST, false><<<grid, kThreads, kSmem, s>>>(a, z); break;
      case ROW_LAST * 2 + 1: bpm_row_kernel<C, ROW_LAST, true><<<grid, kThreads, kSmem, s>>>(a, z); break;
      case ROW_INV_ACC * 2: bpm_row_kernel<C, ROW_INV_ACC, false><<<grid, kThreads, kSmem, s>>>(a, z); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }

  static cudaError_t col(int mode, int grid, const StepArgs& a, int z, cudaStream_t s) {
    if (mode == COL_PROP) bpm_col_kernel<C, COL_PROP><<<grid, kThreads, kSmem, s>>>(a, z);
    else if (mode == COL_FOCUS) bpm_col_kernel<C, COL_FOCUS><<<grid, kThreads, kSmem, s>>>(a, z);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
  }

  static cudaError_t light_sheet(int grid, const StepArgs& a, double w0, double xc, cudaStream_t s) {
    bpm_light_sheet_kernel<C><<<grid, kThreads, kLineSmem, s>>>(a, w0, xc);
    return cudaGetLastError();
  }

  static LenOps make(int n, int sched, int schedules, int is_default) {
    LenOps o;
    o.n = n;
    o.sched = sched;
    o.schedules = schedules;
    o.is_default = is_default;
    o.T = C::T;
    o.NG = C::NG;
    o.four_step = C::FS_N1 > 0;
    o.tw_count = cfg_twiddles<C>();
    o.smem = kSmem;
    o.line_smem = kLineSmem;
    if constexpr (C::kLoop) {
      o.loop = 1;
      o.loop_radix = C::E::R;
      o.loop_passes = C::E::NP;
    } else {
      o.nf = C::F::Rad::count;
      o.ni = C::I::Rad::count;
      for (int i = 0; i < o.nf && i < 4; ++i) o.rf[i] = C::F::Rad::at(i);
      for (int i = 0; i < o.ni && i < 4; ++i) o.ri[i] = C::I::Rad::at(i);
    }
    o.init = &init;
    o.twiddles = &cfg_twiddles_host<C>;
    o.row = &row;
    o.col = &col;
    o.light_sheet = &light_sheet;
    return o;
  }
};

template <class P>
struct PairImpl {
  using CR = typename P::CR;
  using CC = typename P::CC;

  // rows' tables (forward, inverse), then the columns' (forward, inverse,
  // four-step); one copy when rows and columns share a configuration
  static void twiddles(std::vector<float2>& v) {
    cfg_twiddles_host<CR>(v);
    if constexpr (!P::kSame) {
      v.resize(P::TW_ROW);
      cfg_twiddles_host<CC>(v);
    }
  }

  static PairOps make(int sched, int row_sched, int col_sched) {
    PairOps o;
    o.nx = P::NX;
    o.ny = P::NY;
    o.sched = sched;
    o.row_sched = row_sched;
    o.col_sched = col_sched;
    o.row_ng = CR::NG;
    o.col_ng = CC::NG;
    o.four_step = CC::FS_N1 > 0;
    o.col_hs = CC::HS;
    o.tw_count = P::TW_TOTAL;
    o.smem_base = pair_smem_bytes<P>();
    o.kernel[0] = (const void*)bpm_persistent_kernel<P, false>;
    o.kernel[1] = (const void*)bpm_persistent_kernel<P, true>;
    o.twiddles = &twiddles;
    return o;
  }
};

// a length in schedule S (square grids of it use the same schedule for rows
// and columns)
template <int N, int S>
void add_length(OpsRegistry& r) {
  r.lens.push_back(LenImpl<Cfg<N, S>>::make(N, S, kSchedules(N), kDefaultSchedule(N) == S));
  r.pairs.push_back(PairImpl<Pair<Cfg<N, S>, Cfg<N, S>>>::make(S, S, S));
}

// a rectangular grid: rows of length NX and columns of length NY, each in the
// default schedule of its length
template <int NX, int NY>
void add_grid(OpsRegistry& r) {
  constexpr int SR = kDefaultSchedule(NX), SC = kDefaultSchedule(NY);
  r.pairs.push_back(PairImpl<Pair<Cfg<NX, SR>, Cfg<NY, SC>>>::make(0, SR, SC));
}

}  // namespace bpmk
