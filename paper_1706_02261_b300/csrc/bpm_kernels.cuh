// bpm_kernels.cuh - device side of the split-step beam-propagation library.
//
// A "team" of CTAs owns one field of ny rows x nx columns of complex floats
// that lives in global memory (L2-resident: 8 MiB at 1024 x 1024).  Each slice
// of the method is two half-steps, each consuming the other's output:
//
//   column half-step  (CTA owns a block of columns):
//       stage its columns in shared memory, FFT_y, multiply by the propagator
//       column H^T[kx][:], inverse FFT_y, write the columns back;
//   row half-step     (CTA owns a block of rows):
//       inverse FFT_x, phase screen exp(i k0 dn dz) from the FP16 dn row,
//       |E|^2 to the intensity volume, then the forward FFT_x of the next
//       slice (or the FP64 carrier on the last slice), write the row back.
//
// The forward FFT_x of the first slice is a row half-step of its own.  Row
// and column transforms run in registers (see fft.cuh) with one shared-memory
// exchange per radix pass.  The 2D DFT needs all rows before any column, so
// the field crosses between all CTAs twice per slice; in the persistent kernel
// each crossing is a tagged exchange (every element carries the parity of the
// half-step that wrote it, and consumers poll their own elements) rather than
// a team barrier followed by the loads.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "bpm_args.cuh"
#include "fft.cuh"

namespace bpmk {

// Per-length transform configuration.  Two engines:
//  - LoopCfg: N = R^P with one radix R; one pass function (LoopFFT) and the
//    inverse by conjugation, so a half-step is a loop over 2P passes with the
//    pointwise operation (propagator or screen) in the middle, rolled (one
//    compact copy of the pass) or unrolled (U; every configuration here).
//  - GroupCfg: mixed radices (products with 3, or 2^7) through the unrolled
//    GroupFFT with separate forward and inverse schedules.
// Both expose: T threads per row, the register layouts L(R0) (natural order,
// forward input / inverse output) and L(RL) (spectrum order, forward output /
// inverse input), the shared-memory index map f, the group stride GS (chosen
// so that FFT exchanges and column staging are free of bank conflicts for the
// power-of-two sizes) and the twiddle table lengths.  A group of T threads
// holds one row or column; groups wider than a warp (T = 64) synchronise with
// the named barrier 1 + group index.
template <int N_, int T_, int GS_>
struct CfgBase {
  static constexpr int N = N_, T = T_, GS = GS_;
  static constexpr int PTS = N_ / T_;
  static constexpr int NG = kThreads / T_;   // row/column groups per CTA
  static_assert(NG * T_ == kThreads, "groups must tile the CTA");
  static_assert(T_ <= 32 || NG <= 15, "groups wider than a warp use named barriers 1..15");
  // four-step column transform (FourStepCfg): off by default
  static constexpr int FS_N1 = 0, FS_SA = 0, FS_SC = 0, TW4 = 0;
  static constexpr int BUFLEN = NG * GS_;   // float2 of the group / exchange buffers
  static constexpr int HS = N_;             // row stride of the staged propagator columns
  __device__ __forceinline__ static int group() { return threadIdx.x / T_; }
  __device__ __forceinline__ static int lane() { return threadIdx.x % T_; }
  __device__ __forceinline__ static int bar(int gid) { return T_ > 32 ? 1 + gid : 0; }
};

template <int N_, int T_, int R_, int PAD_, int GS_, bool U_ = false>
struct LoopCfg : CfgBase<N_, T_, GS_> {
  using E = LoopFFT<N_, T_, R_, PAD_, U_>;
  static constexpr bool kLoop = true;
  static constexpr int R0 = R_, RL = R_;
  static constexpr int TWF = E::TW, TWI = 0;
  static_assert(GS_ >= E::BUF, "group stride too small");
  __device__ __forceinline__ static int f(int i) { return E::f(i); }
  __device__ __forceinline__ static void fwd(float2* v, float2* buf, const float2* twf, const float2*, int t,
                                             int bar = 0) {
    E::run_fwd(v, buf, twf, t, bar);
  }
  __device__ __forceinline__ static void inv(float2* v, float2* buf, const float2* twf, const float2*, int t,
                                             int bar = 0) {
    E::run_inv(v, buf, twf, t, bar);
  }
  // inverse, mid(v) on natural-order data, forward: one pass loop
  template <class Mid>
  __device__ __forceinline__ static void inv_mid_fwd(float2* v, float2* buf, const float2* twf,
                                                     const float2*, int t, Mid&& mid, int bar = 0) {
    conj_all(v, E::PTS);
    pass_loop<U_, 2 * E::NP>([&](int q) {
      if (q == E::NP) {
        conj_all(v, E::PTS);
        mid(v);
      }
      E::pass(q < E::NP ? q : q - E::NP, v, buf, twf, t, bar);
    });
  }
  // forward, mid(v) on spectrum-order data, inverse: one pass loop
  template <class Mid>
  __device__ __forceinline__ static void fwd_mid_inv(float2* v, float2* buf, const float2* twf,
                                                     const float2*, int t, Mid&& mid, int bar = 0) {
    pass_loop<U_, 2 * E::NP>([&](int q) {
      if (q == E::NP) {
        mid(v);
        conj_all(v, E::PTS);
      }
      E::pass(q < E::NP ? q : q - E::NP, v, buf, twf, t, bar);
    });
    conj_all(v, E::PTS);
  }
  // The propagation step's hand-off from the column to the row half-step
  // carries conjugated data, so that the conjugations around the inverse
  // transforms fold into the neighbouring products.  Both half-steps are then
  // NP forward passes, mid, NP forward passes: on the column side mid returns
  // the conjugate of its product (the inverse of it is left conjugated for the
  // row side); on the row side the first passes take the conjugated spectrum,
  // so mid receives the conjugate of the inverse and returns the plain product
  // for the forward transform.
  template <class Mid>
  __device__ __forceinline__ static void fwd_mid_fwd(float2* v, float2* buf, const float2* twf,
                                                     const float2*, int t, Mid&& mid, int bar = 0) {
    pass_loop<U_, 2 * E::NP>([&](int q) {
      if (q == E::NP) mid(v);
      E::pass(q < E::NP ? q : q - E::NP, v, buf, twf, t, bar);
    });
  }
  // conjugated data in, conjugate of the inverse out
  __device__ __forceinline__ static void inv_c(float2* v, float2* buf, const float2* twf, const float2*, int t,
                                               int bar = 0) {
    E::run_fwd(v, buf, twf, t, bar);
  }
};

template <int N_, int T_, int GS_, class F_, class I_>
struct GroupCfg : CfgBase<N_, T_, GS_> {
  using F = F_;
  using I = I_;
  static constexpr bool kLoop = false;
  static constexpr int R0 = F::R0, RL = F::RL;
  static constexpr int TWF = F::TW, TWI = I::TW;
  static_assert(GS_ >= F::BUF && GS_ >= I::BUF, "group stride too small");
  static_assert(F::RL == I::R0 && I::RL == F::R0, "inverse must reverse the radices");
  __device__ __forceinline__ static int f(int i) { return F::f(i); }
  __device__ __forceinline__ static void fwd(float2* v, float2* buf, const float2* twf, const float2*, int t,
                                             int bar = 0) {
    F::run(v, buf, twf, t, bar);
  }
  __device__ __forceinline__ static void inv(float2* v, float2* buf, const float2*, const float2* twi, int t,
                                             int bar = 0) {
    I::run(v, buf, twi, t, bar);
  }
  template <class Mid>
  __device__ __forceinline__ static void inv_mid_fwd(float2* v, float2* buf, const float2* twf,
                                                     const float2* twi, int t, Mid&& mid, int bar = 0) {
    I::run(v, buf, twi, t, bar);
    mid(v);
    F::run(v, buf, twf, t, bar);
  }
  template <class Mid>
  __device__ __forceinline__ static void fwd_mid_inv(float2* v, float2* buf, const float2* twf,
                                                     const float2* twi, int t, Mid&& mid, int bar = 0) {
    F::run(v, buf, twf, t, bar);
    mid(v);
    I::run(v, buf, twi, t, bar);
  }
};

// Columns of N = N1 * N1 points as a four-step transform (N1 threads per
// column, NG = kThreads / N1 columns per round): thread (a, c), a =
// threadIdx / NG and c = threadIdx % NG, holds y = a + N1 b of column c in
// v[b].  A forward transform is an N1-point DFT over b in registers, the
// twiddle W_N^(a k), an exchange through shared memory (row a of column c's
// N1 x N1 block written, column a read), and a second N1-point DFT; its
// output X[a + N1 k] is in v[k], the same layout as the input, so the
// propagator multiply and the inverse (by conjugation) follow in registers.
// Global loads and stores go straight to registers: per warp instruction,
// rows a .. a + 32/NG - 1 of NG adjacent columns (64-byte segments at
// N1 = 32).  A 64-bit shared-memory access is served per half-warp, whose 16
// lanes hold NG columns c and 16/NG rows a, so the strides make c SC + a SA
// distinct modulo 16 float2 (16 bank pairs): a row of the block SA = 1 and a
// column block SC = 16 / NG (mod 16) for both the row writes and the column
// reads; the staged propagator columns use the row stride HS = N + 16 / NG.
template <class Base, int N1>
struct FourStepCfg : Base {
  static_assert(N1 * N1 == Base::N && N1 * Base::NG == kThreads && Base::NG <= 16,
                "four-step layout needs N = N1^2, N1 NG = kThreads, NG <= 16");
  static constexpr int FS_N1 = N1;
  static constexpr int FS_SA = (N1 + 15) / 16 * 16 + 1;
  static constexpr int FS_SC = N1 * FS_SA + ((16 / Base::NG) % 16 - (N1 * FS_SA) % 16 + 16) % 16;
  static constexpr int TW4 = Base::N;       // W_N^(a k) at [k/2][a][k%2]
  static constexpr int BUFLEN = Base::NG * FS_SC > Base::NG * Base::GS ? Base::NG * FS_SC : Base::NG * Base::GS;
  static constexpr int HS = Base::N + 16 / Base::NG;
};

using Rad8x16 = Radices<8, 16>;
using Rad16x8 = Radices<16, 8>;
using Rad8x8x3 = Radices<8, 8, 3>;
using Rad3x8x8 = Radices<3, 8, 8>;
using Rad8x8x6 = Radices<8, 8, 6>;
using Rad6x8x8 = Radices<6, 8, 8>;
using Rad8x8x4 = Radices<8, 8, 4>;
using Rad4x8x8 = Radices<4, 8, 8>;

// Cfg<N, S>: transform schedule S of length N (S = 0 the default; the other
// schedules of a length are alternatives that bpm_autotune times for
// single-field square plans, kSchedules(N) of them).
template <int N, int S = 0>
struct Cfg;
template <> struct Cfg<64> : LoopCfg<64, 8, 8, 8, 73, true> {};
template <> struct Cfg<96> : GroupCfg<96, 8, 109, GroupFFT<96, 8, 8, -1, Radices<4, 4, 6>>, GroupFFT<96, 8, 8, +1, Radices<6, 4, 4>>> {};
template <> struct Cfg<128> : GroupCfg<128, 8, 145, GroupFFT<128, 8, 8, -1, Rad8x16>, GroupFFT<128, 8, 16, +1, Rad16x8>> {};
template <> struct Cfg<192> : GroupCfg<192, 8, 219, GroupFFT<192, 8, 8, -1, Rad8x8x3>, GroupFFT<192, 8, 8, +1, Rad3x8x8>> {};
// 256 and 512: one row per warp (32 threads, 8 or 16 points each), so a
// single field spreads over 32 or 64 CTAs (about 1.4x and 1.7x shorter slices
// than two rows per warp); schedule 0 of 512 is the radix-8 loop; strides from
// the half-warp bank model.  The radix loops (64, 256 schedule 2, 512
// schedule 0, 1024) are unrolled: with the tagged exchange their pass-index
// branches and twiddle address arithmetic cost more than the larger code
// (slices 13 % shorter at 64^2, 12 % at 512^2, 8 % at 256^2, 6 % at 1024^2;
// the batched schedule sets 0 and 2 6 % and 1 % shorter)
template <> struct Cfg<256> : GroupCfg<256, 32, 274, GroupFFT<256, 32, 16, -1, Rad8x8x4>, GroupFFT<256, 32, 16, +1, Rad4x8x8>> {};
template <> struct Cfg<384> : GroupCfg<384, 16, 409, GroupFFT<384, 16, 16, -1, Rad8x8x6>, GroupFFT<384, 16, 16, +1, Rad6x8x8>> {};
template <> struct Cfg<512> : LoopCfg<512, 32, 8, 16, 546, true> {};
template <> struct Cfg<768> : GroupCfg<768, 32, 818, GroupFFT<768, 32, 16, -1, Radices<8, 8, 12>>, GroupFFT<768, 32, 16, +1, Radices<12, 8, 8>>> {};
template <> struct Cfg<1024> : FourStepCfg<LoopCfg<1024, 32, 32, 32, 1058, true>, 32> {};
// 1536 and 2048: two warps per row or column (64 threads, 24 or 32 points
// each), synchronised by a named barrier per group
template <> struct Cfg<1536> : GroupCfg<1536, 64, 1634, GroupFFT<1536, 64, 16, -1, Radices<8, 8, 24>>, GroupFFT<1536, 64, 16, +1, Radices<24, 8, 8>>> {};
template <> struct Cfg<2048> : GroupCfg<2048, 64, 2178, GroupFFT<2048, 64, 16, -1, Radices<16, 16, 8>>, GroupFFT<2048, 64, 16, +1, Radices<8, 16, 16>>> {};

// Alternative schedules (single-field square plans; bpm_autotune keeps the
// fastest): 512 as unrolled 8 x 8 x 8 or 16 x 16 x 2 passes with separate
// inverse schedules, 256 with the pass order reversed or as the rolled
// radix-16 loop on two rows per warp, 1024 with its columns staged through
// shared memory like the rows instead of the four-step register layout.
template <> struct Cfg<512, 1> : GroupCfg<512, 32, 546, GroupFFT<512, 32, 16, -1, Radices<8, 8, 8>>,
                                          GroupFFT<512, 32, 16, +1, Radices<8, 8, 8>>> {};
template <> struct Cfg<512, 2> : GroupCfg<512, 32, 546, GroupFFT<512, 32, 16, -1, Radices<16, 16, 2>>,
                                          GroupFFT<512, 32, 16, +1, Radices<2, 16, 16>>> {};
template <> struct Cfg<256, 1> : GroupCfg<256, 32, 274, GroupFFT<256, 32, 16, -1, Rad4x8x8>, GroupFFT<256, 32, 16, +1, Rad8x8x4>> {};
template <> struct Cfg<256, 2> : LoopCfg<256, 16, 16, 16, 273, true> {};
template <> struct Cfg<1024, 1> : LoopCfg<1024, 32, 32, 32, 1058, true> {};

// number of schedules of length n (Cfg<n, 0> .. Cfg<n, kSchedules(n) - 1>)
__host__ __device__ constexpr int kSchedules(int n) { return n == 256 || n == 512 ? 3 : (n == 1024 ? 2 : 1); }
// schedule a single-field plan starts with: the fastest measured on a B300
// (us per slice with the intensity volume, tagged exchange: 256^2 4.48 /
// 4.43 / 5.75, 512^2 7.57 / 7.54 / 7.28, 1024^2 10.6 / 13.5); batched plans
// take schedule sets instead (bpm_autotune); the rows and columns of a
// rectangular grid take the default of their own length
__host__ __device__ constexpr int kDefaultSchedule(int n) { return n == 512 ? 2 : 0; }

// One grid's transforms: rows of length NX = CR::N (ny of them), columns of
// length NY = CC::N (nx of them).  Shared memory of the persistent kernel
// holds the row tables (forward, inverse), then the column tables (forward,
// inverse, four-step); a square grid whose rows and columns share one
// configuration keeps one copy.
template <class CR_, class CC_>
struct Pair {
  using CR = CR_;
  using CC = CC_;
  static constexpr int NX = CR::N, NY = CC::N;
  static constexpr bool kSame = std::is_same<CR_, CC_>::value;
  static constexpr int TW_ROW = CR::TWF + CR::TWI;
  static constexpr int TW_COL_OFF = kSame ? 0 : TW_ROW;   // column tables (forward, inverse, four-step)
  static constexpr int TW_TOTAL = kSame ? CR::TWF + CR::TWI + CR::TW4 : TW_ROW + CC::TWF + CC::TWI + CC::TW4;
  static constexpr int BUFLEN = CR::BUFLEN > CC::BUFLEN ? CR::BUFLEN : CC::BUFLEN;
};

// shared memory of the half-step kernels (one length): twiddle tables, then the buffers
template <class C>
__host__ __device__ constexpr size_t cfg_smem_bytes() {
  return sizeof(float2) * (size_t)(C::TWF + C::TWI + C::TW4 + C::BUFLEN);
}
template <class C>
__host__ __device__ constexpr int cfg_twiddles() {
  return C::TWF + C::TWI + C::TW4;
}
// ... and of the persistent kernel of a grid, before its staging buffers
template <class P>
__host__ __device__ constexpr size_t pair_smem_bytes() {
  return sizeof(float2) * (size_t)(P::TW_TOTAL + P::BUFLEN);
}
// exp(i x) for the phase screen: the Taylor series of sin and cos evaluated
// by Horner's rule in x^2 (branch free), for |x| <= pi/4 truncated after x^11
// and x^12 (truncation below 1e-11), with a shorter form for |x| <= 1/8
// below; larger arguments use sincosf.  Callers pick the evaluation once per
// warp (phasor_range) so that the loop over a row's elements has no
// per-element branch and its independent elements can interleave.
constexpr float kPhasorPolyMax = 0.785398163f;

__device__ __forceinline__ float2 unit_phasor_poly(float x) {
  const float x2 = x * x;
  const float ps = fmaf(fmaf(fmaf(fmaf(x2, -2.50521084e-8f, 2.75573192e-6f), x2, -1.98412698e-4f), x2,
                             8.33333333e-3f),
                        x2, -1.66666667e-1f);
  const float s = fmaf(ps, x2 * x, x);
  const float c = fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(x2, 2.08767570e-9f, -2.75573192e-7f), x2, 2.48015873e-5f), x2,
                                      -1.38888889e-3f),
                                 x2, 4.16666667e-2f),
                            x2, -0.5f),
                       x2, 1.0f);
  return make_float2(c, s);
}

constexpr float kPhasorTinyMax = 0.125f;

// The screen evaluates two phases at once with the packed two-lane FP32
// operations of sm_100 and later (lane pair = two elements of a row): cos and
// sin of x.x and x.y, returned as the pairs (cos, cos) and (sin, sin).
// unit_phasor_tiny2 takes |x| <= 1/8 (Taylor series of sin and cos truncated
// after x^5 and x^6: truncation below 1e-10, k0 |dn| dz <= 1/8 covers index
// steps up to 0.06 at 0.1625 um slices and 0.5 um light); unit_phasor_poly2
// is unit_phasor_poly on two lanes.
__device__ __forceinline__ float2 pair(float v) { return make_float2(v, v); }

__device__ __forceinline__ float2 unit_phasor_tiny(float x) {
  const float x2 = x * x;
  const float s = fmaf(fmaf(x2, 8.33333333e-3f, -1.66666667e-1f), x2 * x, x);
  const float c = fmaf(fmaf(fmaf(x2, -1.38888889e-3f, 4.16666667e-2f), x2, -0.5f), x2, 1.0f);
  return make_float2(c, s);
}

__device__ __forceinline__ void unit_phasor_tiny2(float2 x, float2& c, float2& s) {
  const float2 x2 = __fmul2_rn(x, x);
  const float2 ps = __ffma2_rn(x2, pair(8.33333333e-3f), pair(-1.66666667e-1f));
  s = __ffma2_rn(ps, __fmul2_rn(x2, x), x);
  c = __ffma2_rn(__ffma2_rn(__ffma2_rn(x2, pair(-1.38888889e-3f), pair(4.16666667e-2f)), x2, pair(-0.5f)), x2,
                 pair(1.0f));
}

__device__ __forceinline__ void unit_phasor_poly2(float2 x, float2& c, float2& s) {
  const float2 x2 = __fmul2_rn(x, x);
  float2 ps = __ffma2_rn(x2, pair(-2.50521084e-8f), pair(2.75573192e-6f));
  ps = __ffma2_rn(ps, x2, pair(-1.98412698e-4f));
  ps = __ffma2_rn(ps, x2, pair(8.33333333e-3f));
  ps = __ffma2_rn(ps, x2, pair(-1.66666667e-1f));
  s = __ffma2_rn(ps, __fmul2_rn(x2, x), x);
  float2 pc = __ffma2_rn(x2, pair(2.08767570e-9f), pair(-2.75573192e-7f));
  pc = __ffma2_rn(pc, x2, pair(2.48015873e-5f));
  pc = __ffma2_rn(pc, x2, pair(-1.38888889e-3f));
  pc = __ffma2_rn(pc, x2, pair(4.16666667e-2f));
  pc = __ffma2_rn(pc, x2, pair(-0.5f));
  c = __ffma2_rn(pc, x2, pair(1.0f));
}

__device__ __forceinline__ float2 unit_phasor_libm(float x) {
  float s, c;
  sincosf(x, &s, &c);
  return make_float2(c, s);
}
__device__ __forceinline__ void unit_phasor_libm2(float2 x, float2& c, float2& s) {
  sincosf(x.x, &s.x, &c.x);
  sincosf(x.y, &s.y, &c.y);
}

// exp(i x) for any moderate |x| without a branch: Cody-Waite reduction
// x = q pi/2 + r with q = rint(2x/pi) and pi/2 split into a float head and
// tail, the Taylor polynomial of unit_phasor_poly on |r| <= pi/4, and the
// rotation by i^q.  Accurate to FP32 rounding for |x| up to about 1e5.
__device__ __forceinline__ float2 unit_phasor_reduced(float x) {
  constexpr float kTwoOverPi = 0.636619772f;
  constexpr float kHalfPiHi = 1.57079637f;          // float nearest pi/2
  constexpr float kHalfPiLo = -4.37113883e-8f;      // pi/2 - kHalfPiHi
  const float q = rintf(x * kTwoOverPi);
  const float r = fmaf(-q, kHalfPiLo, fmaf(-q, kHalfPiHi, x));
  const float2 e = unit_phasor_poly(r);
  const int k = (int)q & 3;
  const float c = (k & 1) ? e.y : e.x, sn = (k & 1) ? e.x : e.y;
  return make_float2((k == 1 || k == 2) ? -c : c, (k & 2) ? -sn : sn);
}

// The evaluation every lane of the warp can use, from each lane's largest
// |screen phase|: 0 the short polynomial, 1 the long one, 2 sincosf (NaN
// index values keep a polynomial; they are reported separately).
__device__ __forceinline__ int phasor_range(float max_abs_phase) {
  if (__all_sync(0xffffffffu, !(max_abs_phase > kPhasorTinyMax))) return 0;
  return __all_sync(0xffffffffu, !(max_abs_phase > kPhasorPolyMax)) ? 1 : 2;
}

// Per-CTA shared-memory copies used by the half-steps (nullptr = use global).
struct Stage {
  const float2* h = nullptr;   // propagator columns [col - c0][ky]
  const __half* dn = nullptr;  // index rows of the current slice [row - r0][x]
};

// ---------------------------------------------------------------------------
// memory helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// --- tagged exchange (persistent kernel; batched teams of small instances) --
// Between the half-steps of a slice the field crosses from every CTA of the
// team to every other one through L2.  Instead of a team barrier before each crossing (a
// release fence, an arrival add, a poll, then the loads: four L2 latencies in
// a row), every element carries the parity of the half-step that wrote it in
// the lowest mantissa bit of its real part, and each consumer polls the
// elements it needs: row half-steps write 0, column half-steps write 1.  An
// element is one 64-bit access (single-copy atomic), so a value with the
// expected bit is the new value whole.  The only older value a consumer can
// find at a location is its own write of the previous half-step (the same
// thread reads and writes the same positions in every half-step of its kind,
// and every half-step writes every element), which carries the other parity.
// Nothing else crosses between CTAs during the slice loop (the propagator,
// twiddles and index rows are read only), so no fence is needed; one barrier
// with release/acquire semantics after the entrance field's forward FFT_x
// (tag 0) makes it visible over whatever the buffer held before.  Forcing the
// bit moves the real part by at most one unit in the last place per crossing.
__device__ __forceinline__ void st_tagged(float2* p, float2 v, unsigned tag) {
  const unsigned long long b =
      ((unsigned long long)__float_as_uint(v.y) << 32) | ((__float_as_uint(v.x) & ~1u) | tag);
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b) : "memory");
}
__device__ __forceinline__ float2 ld_tagged(const float2* p) {
  unsigned long long b;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(b) : "l"(p));
  return make_float2(__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32)));
}

// --- bulk asynchronous copies (TMA engine, 1D) and mbarriers ---------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared, completion counted on mbarrier m (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, unsigned bytes, uint64_t* m) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_addr(m))
      : "memory");
}

// Bounded wait for an mbarrier phase: gives up after timeout_ns, records
// kDevErrTimeout and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* m, unsigned parity, const StepArgs& a) {
  if (mbar_try_wait(m, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  while (!mbar_try_wait(m, parity)) {
    if (global_timer_ns() - t0 > a.timeout_ns) {
      atomicCAS(a.err, 0, kDevErrTimeout);
      return false;
    }
  }
  return true;
}

// Team barrier over all CTAs of a cooperative grid.  Arrival is a release
// add on a counter that the host zeroes before the launch; the wait polls it
// with acquire loads.  The wait is bounded by timeout_ns (global timer): when
// it runs out, or another CTA has recorded an error, the CTA records
// kDevErrTimeout (first error wins) and the caller leaves the kernel.
__device__ __forceinline__ bool team_barrier(const StepArgs& a, unsigned& epoch, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    const unsigned target = epoch * gridDim.x + a.bar_extra;
    red_release_gpu(a.bar, 1u);
    int ok = 1;
    const unsigned long long t0 = global_timer_ns();
    for (;;) {
      unsigned v = ld_acquire_gpu(a.bar);
      if ((int)(v - target) >= 0) break;
      if (ld_volatile(a.err) != 0) {
        ok = 0;
        break;
      }
      if (global_timer_ns() - t0 > a.timeout_ns) {
        atomicCAS(a.err, 0, kDevErrTimeout);
        ok = 0;
        break;
      }
    }
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// Loads P elements of the tagged field, v[slot(i)] from ptr(slot(i)) in issue
// order i, then reloads the ones that do not carry the tag WANT until all do.
// Each round trip re-reads only the groups that still miss an element, right
// after the previous round's values arrive: the consumer's reaction time is
// on the critical path of the slice (a back-off of 100 ns between rounds, or
// polling one missing element before reloading the rest, measured 40 % and
// 11 % slower at 1024 x 1024).  The wait is bounded like the team barrier:
// when timeout_ns runs out, or another CTA has recorded an error, it records
// kDevErrTimeout (first error wins) and returns false, leaving whatever was
// read in v (the caller finishes its half-step on it, so that the CTA's
// barriers stay matched, and then leaves).
template <unsigned WANT, int P, class Slot, class Ptr>
__device__ __forceinline__ bool load_tagged(float2* v, Slot&& slot, Ptr&& ptr, const StepArgs& a) {
#pragma unroll
  for (int i = 0; i < P; ++i) {
    const int k = slot(i);
    v[k] = ld_tagged(ptr(k));
  }
  // all tags equal to WANT: the AND of the words has the bit (WANT 1), or
  // their OR lacks it (WANT 0); three-input logic folds two words per step
  unsigned acc = WANT ? ~0u : 0u;
#pragma unroll
  for (int k = 0; k < P; ++k) acc = WANT ? (acc & __float_as_uint(v[k].x)) : (acc | __float_as_uint(v[k].x));
  if ((acc & 1u) == WANT) return true;
  const unsigned long long t0 = global_timer_ns();
  for (unsigned round = 1;; ++round) {
    bool again = false;
    // groups of four elements: one test per group, the whole group reloaded
    // when any of it misses (fewer instructions per round than testing each)
    constexpr int GQ = P % 4 == 0 ? 4 : 1;
#pragma unroll
    for (int g = 0; g < P; g += GQ) {
      unsigned gacc = WANT ? ~0u : 0u;
#pragma unroll
      for (int j = 0; j < GQ; ++j) {
        const unsigned w = __float_as_uint(v[slot(g + j)].x);
        gacc = WANT ? (gacc & w) : (gacc | w);
      }
      if ((gacc & 1u) != WANT) {
#pragma unroll
        for (int j = 0; j < GQ; ++j) {
          const int k = slot(g + j);
          v[k] = ld_tagged(ptr(k));
        }
        again = true;
      }
    }
    if (!again) return true;
    // the limit and the error word are checked every eighth round (each
    // check adds to the round's latency: 0.5 % shorter slices at 1024 x 1024)
    if ((round & 7u) == 0 && (global_timer_ns() - t0 > a.timeout_ns || ld_volatile(a.err) != 0)) {
      atomicCAS(a.err, 0, kDevErrTimeout);
      return false;
    }
  }
}

// First-order correction of the propagator to slice z's mean index (reading
// B): w[k] *= exp(i dl g(k)), k < count, with g(k) read by gk(k).  The phase
// grows without bound towards the evanescent cut (g ~ 1 / kz0) and every
// column holds a few such components, so a per-warp choice would always fall
// to sincosf; the branch-free reduced evaluation serves all elements.
template <int COUNT, class GK>
__device__ __forceinline__ void adapt_multiply(float2* w, float dl, GK&& gk) {
#pragma unroll
  for (int k = 0; k < COUNT; ++k) w[k] = cmul(w[k], unit_phasor_reduced(dl * gk(k)));
}

// ---------------------------------------------------------------------------
// half-steps
// ---------------------------------------------------------------------------

// Loads in the order the first radix-R pass consumes them, stores in the
// order the last one produces them (dft_input_order / dft_output_order).
template <int N, int T, int R>
__device__ __forceinline__ void load_layout(float2* v, const float2* __restrict__ src, int t) {
#pragma unroll
  for (int i = 0; i < N / T; ++i) {
    const int k = (i / R) * R + dft_input_order<R>(i % R);
    v[k] = __ldcg(src + layout_index<N, T, R>(k, t));
  }
}
template <int N, int T, int R>
__device__ __forceinline__ void store_layout(const float2* v, float2* dst, int t) {
#pragma unroll
  for (int i = 0; i < N / T; ++i) {
    const int k = (i / R) * R + dft_output_order<R>(i % R);
    __stcg(dst + layout_index<N, T, R>(k, t), v[k]);
  }
}
// ... the same layouts on the tagged field
template <unsigned WANT, int N, int T, int R>
__device__ __forceinline__ bool load_layout_tagged(float2* v, const float2* src, int t, const StepArgs& a) {
  return load_tagged<WANT, N / T>(
      v, [](int i) { return (i / R) * R + dft_input_order<R>(i % R); },
      [&](int k) { return src + layout_index<N, T, R>(k, t); }, a);
}
template <int N, int T, int R>
__device__ __forceinline__ void store_layout_tagged(const float2* v, float2* dst, int t, unsigned tag) {
#pragma unroll
  for (int i = 0; i < N / T; ++i) {
    const int k = (i / R) * R + dft_output_order<R>(i % R);
    st_tagged(dst + layout_index<N, T, R>(k, t), v[k], tag);
  }
}

// Rows [r0, r1) of the team member (rows of length C::N; NYc rows in all, or
// a.ny when NYc is 0); each group of T threads takes one row per round.
// Groups without a row run the transforms on zeros (so that the warp or
// group stays converged for its barriers) and skip all memory traffic.
// TG: the working field is the tagged field of the exchange (rows read the
// column half-step's tag 1 and write tag 0; the last slice's output is
// written plain).  Returns false when a tagged wait gave up.
template <class C, int NYc, int MODE, bool KAPPA = false, bool PK = true, bool TG = false>
__device__ __forceinline__ bool row_half_step(const StepArgs& a, int r0, int r1, int z, float2* s_buf,
                                              const float2* s_twf, const float2* s_twi, bool& bad,
                                              const Stage& st = Stage()) {
  constexpr int N = C::N;
  const int ny = NYc ? NYc : a.ny;
  const int gid = C::group();
  const int t = C::lane();
  const int gbar = C::bar(gid);
  float2* buf = s_buf + gid * C::GS;
  const int rounds = (r1 - r0 + C::NG - 1) / C::NG;
  bool ok = true;
  for (int k = 0; k < rounds; ++k) {
    const int row = r0 + k * C::NG + gid;
    const bool active = row < r1;
    float2 v[C::PTS];
    if constexpr (MODE == ROW_FWD) {
      if (active) load_layout<N, C::T, C::R0>(v, a.ein + (size_t)row * N, t);
      else
#pragma unroll
        for (int q = 0; q < C::PTS; ++q) v[q] = make_float2(0.f, 0.f);
      C::fwd(v, buf, s_twf, s_twi, t, gbar);
      if (active) {
        if constexpr (TG) store_layout_tagged<N, C::T, C::RL>(v, a.work + (size_t)row * N, t, a.tag_stall ? 1u : 0u);
        else store_layout<N, C::T, C::RL>(v, a.work + (size_t)row * N, t);
      }
    } else if constexpr (MODE == ROW_INV_ACC) {
      if (active) load_layout<N, C::T, C::RL>(v, a.work + (size_t)row * N, t);
      else
#pragma unroll
        for (int q = 0; q < C::PTS; ++q) v[q] = make_float2(0.f, 0.f);
      C::inv(v, buf, s_twf, s_twi, t, gbar);
      if (active) {
        float2* dst = a.out + (size_t)row * N;
#pragma unroll
        for (int q = 0; q < C::PTS; ++q) {
          const int x = layout_index<N, C::T, C::R0>(q, t);
          float2 o = v[q];
          if (a.accumulate) o = cadd(o, __ldcg(dst + x));
          __stcg(dst + x, o);
        }
      }
    } else {
      if (active) {
        if constexpr (TG) ok &= load_layout_tagged<1u, N, C::T, C::RL>(v, a.work + (size_t)row * N, t, a);
        else load_layout<N, C::T, C::RL>(v, a.work + (size_t)row * N, t);
      } else {
#pragma unroll
        for (int q = 0; q < C::PTS; ++q) v[q] = make_float2(0.f, 0.f);
      }
      // index values: from the shared-memory copy of this CTA's rows when the
      // slice was prefetched, else fetched from global memory before the
      // inverse transform so that their latency hides behind it
      __half dv[C::PTS];
      if (!st.dn) {
        const __half* dnrow = a.dn + ((size_t)z * ny + (active ? row : r0)) * N;
#pragma unroll
        for (int q = 0; q < C::PTS; ++q) dv[q] = __ldcs(dnrow + layout_index<N, C::T, C::R0>(q, t));
      }
      const __half* sdn = st.dn ? st.dn + (size_t)((active ? row : r0) - r0) * N : nullptr;
      // absorption row (global memory, read once per element with streaming
      // loads), only in the KAPPA instantiation: staging it next to the index
      // rows would move the persistent kernel to the next, larger
      // shared-memory carve-out and shrink L1, which slows the lossless path
      const __half* skap = nullptr;
      if constexpr (KAPPA) skap = a.kappa + ((size_t)z * ny + (active ? row : r0)) * N;
      // |E|^2 goes straight from the registers to the intensity volume with
      // streaming stores (staging the rows in shared memory for one bulk store
      // per CTA measured 3.6 % slower per 1024^2 slice: its proxy fence and
      // CTA barrier sit on the path of every slice)
      float* irow = nullptr;
      if (active && a.inten && z >= a.iz0 && z < a.iz1) irow = a.inten + ((size_t)(z - a.iz0) * ny + row) * N;
      // LoopFFT sizes receive the conjugated spectrum from the column
      // half-step (LoopCfg::fwd_mid_fwd): the screen multiplies conj(w)
      constexpr bool CJ = C::kLoop;
      auto scr = [](float2 w, float2 p) { return CJ ? cmul_conj_in(w, p) : cmul(w, p); };
      // phase screen exp(i k0 dn dz) and |E|^2 on the natural-order field;
      // the evaluation of the phasor (polynomial or sincosf) is chosen once per
      // warp so the element loop is branch free and its elements interleave
      auto screen = [&](float2* w) {
        // index values of this thread's elements: from the shared-memory rows
        // (prefetched) or the registers fetched before the transform
        float dval[C::PTS];
        float mx = 0.f, sum = 0.f;    // fmaxf skips NaN; the sum keeps NaN and inf
#pragma unroll
        for (int q = 0; q < C::PTS; ++q) {
          dval[q] = __half2float(sdn ? sdn[layout_index<N, C::T, C::R0>(q, t)] : dv[q]);
          mx = fmaxf(mx, fabsf(dval[q]));
          sum += dval[q];
        }
        bad |= active && !isfinite(sum);
        // reading B: the screen acts on dn - delta[z] (the slice's mean index
        // step went into the propagator)
        const float off = a.delta ? a.delta[z] : 0.f;
        const float c0 = -a.screen_c * off;
        const int range = phasor_range(a.screen_c * (mx + fabsf(off)));
        // PK: two elements per packed evaluation (single-instance kernels);
        // the batched kernel, whose one instruction stream holds every size,
        // measured faster with the scalar form
        static_assert(!PK || C::PTS % 2 == 0, "the packed screen takes elements in pairs");
        auto body2 = [&](auto phasor2) {
#pragma unroll
          for (int q = 0; q < C::PTS; q += 2) {
            // |E|^2 after the (unit-modulus) screen is |E|^2 before it, to the
            // phasor's rounding; taken first it does not wait for the phasor
            if (irow) {
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const int x = layout_index<N, C::T, C::R0>(q + u, t);
                const float iv = fmaf(w[q + u].x, w[q + u].x, w[q + u].y * w[q + u].y);
                __stcs(irow + x, iv);
              }
            }
            float2 cs, sn;
            phasor2(__ffma2_rn(pair(a.screen_c), make_float2(dval[q], dval[q + 1]), pair(c0)), cs, sn);
            w[q] = scr(w[q], make_float2(cs.x, sn.x));
            w[q + 1] = scr(w[q + 1], make_float2(cs.y, sn.y));
          }
        };
        auto body1 = [&](auto phasor) {
#pragma unroll
          for (int q = 0; q < C::PTS; ++q) {
            const float2 wq = w[q];
            if (irow) {
              const int x = layout_index<N, C::T, C::R0>(q, t);
              const float iv = fmaf(wq.x, wq.x, wq.y * wq.y);
              __stcs(irow + x, iv);
            }
            w[q] = scr(wq, phasor(fmaf(a.screen_c, dval[q], c0)));
          }
        };
        if constexpr (KAPPA) {
          // complex index: exp(i k0 (dn + i kappa) dz) = exp(i k0 dn dz) exp(-k0 kappa dz)
          float ksum = 0.f;
#pragma unroll
          for (int q = 0; q < C::PTS; ++q) {
            const int x = layout_index<N, C::T, C::R0>(q, t);
            const float kv = __half2float(__ldcs(skap + x));
            ksum += kv;
            const float2 e = scr(w[q], unit_phasor_reduced(fmaf(a.screen_c, dval[q], c0)));
            const float att = expf(-a.screen_c * kv);
            w[q] = make_float2(e.x * att, e.y * att);
            if (irow) {
              const float iv = fmaf(w[q].x, w[q].x, w[q].y * w[q].y);
              __stcs(irow + x, iv);
            }
          }
          bad |= active && !isfinite(ksum);
        } else {
          if constexpr (PK) {
            if (range == 0) body2([](float2 ph, float2& c, float2& sn) { unit_phasor_tiny2(ph, c, sn); });
            else if (range == 1) body2([](float2 ph, float2& c, float2& sn) { unit_phasor_poly2(ph, c, sn); });
            else body2([](float2 ph, float2& c, float2& sn) { unit_phasor_libm2(ph, c, sn); });
          } else {
            if (range == 0) body1([](float ph) { return unit_phasor_tiny(ph); });
            else if (range == 1) body1([](float ph) { return unit_phasor_poly(ph); });
            else body1([](float ph) { return unit_phasor_libm(ph); });
          }
        }
      };
      if constexpr (MODE == ROW_LAST) {
        if constexpr (CJ) C::inv_c(v, buf, s_twf, s_twi, t, gbar);
        else C::inv(v, buf, s_twf, s_twi, t, gbar);
        screen(v);
        if (active) {
#pragma unroll
          for (int q = 0; q < C::PTS; ++q) v[q] = cmul(v[q], a.carrier);
          store_layout<N, C::T, C::R0>(v, a.work + (size_t)row * N, t);
        }
      } else {
        if constexpr (CJ) C::fwd_mid_fwd(v, buf, s_twf, s_twi, t, screen, gbar);
        else C::inv_mid_fwd(v, buf, s_twf, s_twi, t, screen, gbar);
        if (active) {
          if constexpr (TG) store_layout_tagged<N, C::T, C::RL>(v, a.work + (size_t)row * N, t, 0u);
          else store_layout<N, C::T, C::RL>(v, a.work + (size_t)row * N, t);
        }
      }
    }
  }
  return ok;
}

// One forward four-step transform of the columns held as in FourStepCfg:
// N1-point DFT over the registers, twiddles W_N^(a k) (tw = pair table + a,
// the pair of k = 2 kp, 2 kp + 1 at stride N1: the NG threads of a row share
// each value), exchange
// (xw: this thread's row of its column block, xr: its column, stride SA),
// N1-point DFT.  Two CTA barriers: the buffer is free before it is written
// (skipped when the caller knows it is: buffer_free), and complete before it
// is read.
template <int N1, int SA>
__device__ __forceinline__ void four_step_fwd(float2* v, const float4* tw, float2* xw, const float2* xr,
                                              bool buffer_free = false) {
  Dft<N1, -1>::run(v);
#pragma unroll
  for (int kp = 0; kp < N1 / 2; ++kp) {
    const float4 w = tw[kp * N1];
    if (kp > 0) v[2 * kp] = cmul(v[2 * kp], make_float2(w.x, w.y));
    v[2 * kp + 1] = cmul(v[2 * kp + 1], make_float2(w.z, w.w));
  }
  if (!buffer_free) __syncthreads();
#pragma unroll
  for (int k = 0; k < N1; ++k) xw[k] = v[k];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < N1; ++j) v[j] = xr[j * SA];
  Dft<N1, -1>::run(v);
}

// Columns [c0, c1) (length C::N; row stride NXc, or a.nx when NXc is 0) by
// four-step transforms (FourStepCfg): load, FFT_y, propagator H^T[col][ky],
// inverse FFT_y (conjugated forward), store, NG columns per round, all in
// registers apart from the two exchanges.
template <class C, int NXc, int FLIP, bool TG = false>
__device__ __forceinline__ bool col_half_step_4s(const StepArgs& a, int c0, int c1, int z, float2* s_buf,
                                                 const float2* s_tw4, const Stage& st) {
  constexpr int N = C::N;
  constexpr int N1 = C::FS_N1, NG = C::NG, SA = C::FS_SA, SC = C::FS_SC;
  const int nx = NXc ? NXc : a.nx;
  const int c = threadIdx.x % NG, ai = threadIdx.x / NG;
  // [k/2][a][k%2] pairs (16-byte aligned: the table follows whole tables)
  const float4* tw = reinterpret_cast<const float4*>(s_tw4) + ai;
  float2* xw = s_buf + c * SC + ai * SA;
  const float2* xr = s_buf + c * SC + ai;
  bool ok = true;
  for (int cb = c0; cb < c1; cb += NG) {
    const int col = cb + c;
    const bool on = col < c1;
    float2 v[N1];
    {
      const float2* src = a.work + (on ? col : c0);
      if constexpr (TG) {
        // a column without data (past c1) reads the first column, whose
        // elements carry the same tag
        ok &= load_tagged<0u, N1>(
            v, [](int i) { return dft_input_order<N1>(i); },
            [&](int b) { return src + (size_t)(ai + N1 * b) * nx; }, a);
      } else {
#pragma unroll
        for (int i = 0; i < N1; ++i) {
          const int b = dft_input_order<N1>(i);
          v[b] = __ldcg(src + (size_t)(ai + N1 * b) * nx);
        }
      }
    }
    // callers with TG put a CTA barrier before the half-step, so the exchange
    // buffer of its first round is free already
    four_step_fwd<N1, SA>(v, tw, xw, xr, TG && cb == c0);
    // conj(X H [exp(i delta G)]): the inverse FFT_y is the forward one of the
    // conjugate, and its conjugated output goes to the row half-step as it is
    if (st.h) {
      const float2* h = st.h + (size_t)((on ? col : c0) - c0) * C::HS + ai;
#pragma unroll
      for (int k = 0; k < N1; ++k) v[k] = cmul_conj_out(v[k], h[N1 * k]);
    } else {
      const float2* h = a.ht + (size_t)(on ? col : c0) * N + ai;
#pragma unroll
      for (int k = 0; k < N1; ++k) v[k] = cmul_conj_out(v[k], __ldg(h + N1 * k));
    }
    if (a.delta) {
      const float* g = a.gt + (size_t)(on ? col : c0) * N + ai;
      adapt_multiply<N1>(v, -a.delta[z], [&](int k) { return __ldg(g + N1 * k); });
    }
    four_step_fwd<N1, SA>(v, tw, xw, xr);
    if (FLIP == 1 || (FLIP == 2 && a.flip_col)) conj_all(v, N1);
    if (on) {
      float2* dst = a.work + col;
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        const int b = dft_output_order<N1>(i);
        if constexpr (TG) st_tagged(dst + (size_t)(ai + N1 * b) * nx, v[b], 1u);
        else __stcg(dst + (size_t)(ai + N1 * b) * nx, v[b]);
      }
    }
  }
  return ok;
}

// Columns [c0, c1) of the team member (length C::N, row stride NXc or a.nx),
// NG columns per round staged in shared memory (column g of the round at
// s_buf + g * GS, index padded like the forward transform's exchange buffer).
// Lengths with a four-step layout take col_half_step_4s for the propagator.
// The propagator step hands the rows conjugated data when the column
// configuration is a rolled loop (LoopCfg::fwd_mid_fwd), and the row
// half-step expects conjugated data when the row configuration is one; when
// the two differ (a rectangular grid) FLIP conjugates the columns' output
// (FLIP 1: always; 2: when a.flip_col is set, for the per-half-step launches).
// TG: the tagged field of the exchange (columns read the row half-step's
// tag 0 and write tag 1); returns false when a tagged wait gave up.
template <class C, int NXc, int MODE, int FLIP = 0, bool TG = false>
__device__ __forceinline__ bool col_half_step(const StepArgs& a, int c0, int c1, int z, float2* s_buf,
                                              const float2* s_twf, const float2* s_twi,
                                              const Stage& st = Stage()) {
  constexpr int N = C::N;
  if constexpr (C::FS_N1 > 0 && MODE == COL_PROP) {
    return col_half_step_4s<C, NXc, FLIP, TG>(a, c0, c1, z, s_buf, s_twi + C::TWI, st);
  }
  bool ok = true;
  const int nx = NXc ? NXc : a.nx;
  const int gid = C::group();
  const int t = C::lane();
  const int gbar = C::bar(gid);
  float2* buf = s_buf + gid * C::GS;
  static_assert(kThreads % C::NG == 0, "");
  constexpr int YSTEP = kThreads / C::NG;
  constexpr int PER = N / YSTEP;
  for (int cb = c0; cb < c1; cb += C::NG) {
    const int nc = min(C::NG, c1 - cb);
    __syncthreads();
    {
      // each thread keeps one column (cc) and walks y; all loads of a chunk
      // are issued before any is consumed
      constexpr int CHUNK = PER % 16 == 0 ? 16 : (PER % 8 == 0 ? 8 : (PER % 4 == 0 ? 4 : 1));
      static_assert(PER % CHUNK == 0, "");
      const int cc = threadIdx.x % C::NG, y0 = threadIdx.x / C::NG;
      const bool on = cc < nc;
      const float2* src = a.work + cb + cc;
#pragma unroll
      for (int c = 0; c < PER; c += CHUNK) {
        float2 tmp[CHUNK];
        if (TG && on) {
          ok &= load_tagged<0u, CHUNK>(
              tmp, [](int i) { return i; }, [&](int i) { return src + (size_t)(y0 + (c + i) * YSTEP) * nx; }, a);
        } else {
#pragma unroll
          for (int i = 0; i < CHUNK; ++i)
            tmp[i] = on ? __ldcg(src + (size_t)(y0 + (c + i) * YSTEP) * nx) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < CHUNK; ++i) s_buf[cc * C::GS + C::f(y0 + (c + i) * YSTEP)] = tmp[i];
      }
    }
    __syncthreads();
    const bool active = gid < nc;
    const int col = cb + gid;
    float2 v[C::PTS];
#pragma unroll
    for (int q = 0; q < C::PTS; ++q)
      v[q] = active ? buf[C::f(layout_index<N, C::T, C::R0>(q, t))] : make_float2(0.f, 0.f);
    group_sync<C::T>(gbar);
    if constexpr (MODE == COL_PROP) {
      const float2* hcol = st.h ? st.h + (size_t)((active ? col : c0) - c0) * C::HS
                                : a.ht + (size_t)(active ? col : c0) * N;
      // LoopFFT sizes hand the row half-step the conjugated inverse
      // (LoopCfg::fwd_mid_fwd): mid returns conj(X H [exp(i delta G)])
      constexpr bool CJ = C::kLoop;
      auto prop = [&](float2* w) {
        auto hm = [](float2 x, float2 h) { return CJ ? cmul_conj_out(x, h) : cmul(x, h); };
        if (st.h) {
#pragma unroll
          for (int q = 0; q < C::PTS; ++q) w[q] = hm(w[q], hcol[layout_index<N, C::T, C::RL>(q, t)]);
        } else {
#pragma unroll
          for (int q = 0; q < C::PTS; ++q) w[q] = hm(w[q], __ldg(hcol + layout_index<N, C::T, C::RL>(q, t)));
        }
        if (a.delta) {
          const float* g = a.gt + (size_t)(active ? col : c0) * N;
          adapt_multiply<C::PTS>(w, CJ ? -a.delta[z] : a.delta[z],
                                 [&](int q) { return __ldg(g + layout_index<N, C::T, C::RL>(q, t)); });
        }
      };
      if constexpr (CJ) C::fwd_mid_fwd(v, buf, s_twf, s_twi, t, prop, gbar);
      else C::fwd_mid_inv(v, buf, s_twf, s_twi, t, prop, gbar);
      if (FLIP == 1 || (FLIP == 2 && a.flip_col)) conj_all(v, C::PTS);
    } else {
      // focusing filter: exp(-i kz zf) / (nx ny) inside the pupil, 0 outside;
      // membership decided in FP64 with the same operation order as the oracle
      const int fx = col < (nx + 1) / 2 ? col : col - nx;
      const double kx = __ddiv_rn(__dmul_rn(6.283185307179586, (double)fx), __dmul_rn((double)nx, a.dx));
      const double ndy = __dmul_rn((double)N, a.dy);
      C::fwd_mid_inv(v, buf, s_twf, s_twi, t, [&](float2* w) {
#pragma unroll
        for (int q = 0; q < C::PTS; ++q) {
          const int ky_i = layout_index<N, C::T, C::RL>(q, t);
          const int fy = ky_i < (N + 1) / 2 ? ky_i : ky_i - N;
          const double ky = __ddiv_rn(__dmul_rn(6.283185307179586, (double)fy), ndy);
          const double kp2 = __dadd_rn(__dmul_rn(kx, kx), __dmul_rn(ky, ky));
          const double kz2 = __dsub_rn(__dmul_rn(a.k0n0, a.k0n0), kp2);
          float2 m = make_float2(0.f, 0.f);
          if (kp2 >= a.kin2 && kp2 <= a.kna2 && kz2 > 0.0) {
            double ph = -sqrt(kz2) * a.zf;
            ph -= 6.283185307179586 * rint(ph * 0.15915494309189535);
            float sn, cs;
            sincosf((float)ph, &sn, &cs);
            const float sc = 1.0f / ((float)nx * (float)N);
            m = make_float2(cs * sc, sn * sc);
          }
          w[q] = cmul(w[q], m);
        }
      }, gbar);
    }
    if (active) {
#pragma unroll
      for (int q = 0; q < C::PTS; ++q) buf[C::f(layout_index<N, C::T, C::R0>(q, t))] = v[q];
    }
    __syncthreads();
    {
      const int cc = threadIdx.x % C::NG, y0 = threadIdx.x / C::NG;
      if (cc < nc) {
        float2* dst = a.work + cb + cc;
#pragma unroll 8
        for (int i = 0; i < PER; ++i) {
          const int y = y0 + i * YSTEP;
          if constexpr (TG) st_tagged(dst + (size_t)y * nx, s_buf[cc * C::GS + C::f(y)], 1u);
          else __stcg(dst + (size_t)y * nx, s_buf[cc * C::GS + C::f(y)]);
        }
      }
    }
  }
  return ok;
}

// count twiddles from global to shared memory (ends with __syncthreads)
__device__ __forceinline__ void load_twiddles(const float2* src, float2* dst, int count) {
  for (int i = threadIdx.x; i < count; i += kThreads) dst[i] = __ldg(src + i);
  __syncthreads();
}

__device__ __forceinline__ void report_bad(const StepArgs& a, bool bad) {
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(a.err, 0, kDevErrNan);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// The whole slice loop in one cooperative launch; gridDim.x CTAs form the team
// (rows split evenly, columns in aligned groups of NG).
// Shared memory: twiddles (rows, columns) | group buffers | [propagator
// columns of this CTA] | [index rows of the current slice].  The index rows
// of slice z are fetched by one bulk copy issued when the column half-step of
// slice z starts, so the HBM read overlaps it; the intensity rows leave the
// row half-step as streaming stores.
template <class P, bool KAPPA = false>
__global__ void __launch_bounds__(kThreads, 1) bpm_persistent_kernel(StepArgs a) {
  using CR = typename P::CR;
  using CC = typename P::CC;
  constexpr int NX = P::NX, NY = P::NY;
  extern __shared__ float4 smem_f4[];
  float2* s_tw = reinterpret_cast<float2*>(smem_f4);
  const float2* s_twr_f = s_tw;                           // row tables
  const float2* s_twr_i = s_tw + CR::TWF;
  const float2* s_twc_f = s_tw + P::TW_COL_OFF;           // column tables
  const float2* s_twc_i = s_twc_f + CC::TWF;
  float2* s_buf = s_tw + P::TW_TOTAL;
  char* s_extra = reinterpret_cast<char*>(s_buf + P::BUFLEN);
  __shared__ int s_flag;
  __shared__ __align__(8) uint64_t s_mbar;
  const int G = gridDim.x, rank = blockIdx.x;
  const int lo = (int)(((long long)rank * NY) / G), hi = (int)(((long long)(rank + 1) * NY) / G);
  const int nrow = hi - lo;
  // columns in whole groups of NG (aligned 64-byte segments at 1024 x 1024):
  // a team larger than NX / NG leaves its last CTAs without columns, while
  // every CTA still takes rows
  const int cper = (NX + G - 1) / G, CB = (cper + CC::NG - 1) / CC::NG * CC::NG;
  const int clo = min(NX, rank * CB), chi = min(NX, clo + CB);
  Stage st;
  {
    size_t off = 0;
    if (a.h_res) {
      st.h = reinterpret_cast<const float2*>(s_extra + off);
      off += ((size_t)a.rmax_c * CC::HS * sizeof(float2) + 15) & ~(size_t)15;
    }
    if (a.dn_stage) {
      st.dn = reinterpret_cast<const __half*>(s_extra + off);
    }
  }
  if (a.h_res) {
    float2* dst = const_cast<float2*>(st.h);
    const float2* src = a.ht + (size_t)clo * NY;
    for (int i = threadIdx.x; i < (chi - clo) * NY; i += kThreads) dst[(i / NY) * CC::HS + i % NY] = __ldg(src + i);
  }
  if (threadIdx.x == 0 && a.dn_stage) mbar_init(&s_mbar, 1);
  load_twiddles(a.tw, s_tw, P::TW_TOTAL);    // ends with __syncthreads
  unsigned epoch = 0, dn_parity = 0;
  bool bad = false, dn_pending = false;
  // the entrance field's forward FFT_x writes the tagged field (tag 0); the
  // one team barrier of the launch makes the first column half-step's reads
  // find it (the field held the previous launch's untagged output before)
  row_half_step<CR, NY, ROW_FWD, false, true, true>(a, lo, hi, a.z_begin, s_buf, s_twr_f, s_twr_i, bad);
  if (!team_barrier(a, epoch, &s_flag)) return;
  for (int zi = a.z_begin; zi < a.z_end; ++zi) {
    const bool last = zi + 1 == a.z_end;
    const int z = a.reverse ? a.z_begin + a.z_end - 1 - zi : zi;     // the slice this step crosses
    if (a.dn_stage && nrow > 0) {
      if (threadIdx.x == 0) {
        const unsigned bytes = (unsigned)((size_t)nrow * NX * sizeof(__half));
        mbar_arrive_expect_tx(&s_mbar, bytes);
        bulk_load(const_cast<__half*>(st.dn), a.dn + ((size_t)z * NY + lo) * NX, bytes, &s_mbar);
      }
      dn_pending = true;
    }
    // the half-steps exchange the field through its tags (no team barrier);
    // a CTA barrier separates their uses of the shared buffers
    bool ok = col_half_step<CC, NX, COL_PROP, (CC::kLoop != CR::kLoop ? 1 : 0), true>(a, clo, chi, z, s_buf,
                                                                                      s_twc_f, s_twc_i, st);
    if (dn_pending) {
      ok = mbar_wait_bounded(&s_mbar, dn_parity, a) && ok;
      dn_parity ^= 1u;
      dn_pending = false;
    }
    if (__syncthreads_or(!ok)) break;
    if (!last) ok = row_half_step<CR, NY, ROW_STEP, KAPPA, true, true>(a, lo, hi, z, s_buf, s_twr_f, s_twr_i, bad, st);
    else ok = row_half_step<CR, NY, ROW_LAST, KAPPA, true, true>(a, lo, hi, z, s_buf, s_twr_f, s_twr_i, bad, st);
    if (__syncthreads_or(!ok)) break;
  }
  // leave no copy in flight: a prefetch abandoned by a failed wait is
  // waited for (bounded)
  if (dn_pending) mbar_wait_bounded(&s_mbar, dn_parity, a);
  report_bad(a, bad);
}

// One half-step per launch (comparison path and input synthesis): rows of
// length C::N (a.ny of them), or columns of length C::N (a.nx of them).
// Shared memory: the length's tables (forward, inverse, four-step) | buffers.
template <class C, int MODE, bool KAPPA = false>
__global__ void __launch_bounds__(kThreads, 1) bpm_row_kernel(StepArgs a, int z) {
  extern __shared__ float4 smem_f4[];
  float2* s_twf = reinterpret_cast<float2*>(smem_f4);
  float2* s_twi = s_twf + C::TWF;
  float2* s_buf = s_twi + C::TWI + C::TW4;
  load_twiddles(a.tw, s_twf, cfg_twiddles<C>());
  const int G = gridDim.x, rank = blockIdx.x;
  const int lo = (int)(((long long)rank * a.ny) / G), hi = (int)(((long long)(rank + 1) * a.ny) / G);
  bool bad = false;
  row_half_step<C, 0, MODE, KAPPA>(a, lo, hi, z, s_buf, s_twf, s_twi, bad);
  if constexpr (MODE == ROW_STEP || MODE == ROW_LAST) report_bad(a, bad);
}

template <class C, int MODE>
__global__ void __launch_bounds__(kThreads, 1) bpm_col_kernel(StepArgs a, int z) {
  extern __shared__ float4 smem_f4[];
  float2* s_twf = reinterpret_cast<float2*>(smem_f4);
  float2* s_twi = s_twf + C::TWF;
  float2* s_buf = s_twi + C::TWI + C::TW4;
  load_twiddles(a.tw, s_twf, cfg_twiddles<C>());
  const int G = gridDim.x, rank = blockIdx.x;
  const int lo = (int)(((long long)rank * a.nx) / G), hi = (int)(((long long)(rank + 1) * a.nx) / G);
  col_half_step<C, 0, MODE, 2>(a, lo, hi, z, s_buf, s_twf, s_twi);
}

// Light sheet: the ky = 0 spectrum line (rows of length C::N), inverse FFT_x
// by group 0, then the row is copied to every y.  Every CTA computes the
// (short) line itself and writes a share of the rows.  Dynamic shared memory:
// cfg_smem_bytes() plus GS float2 for the spectrum line.
template <class C>
__global__ void __launch_bounds__(kThreads, 1) bpm_light_sheet_kernel(StepArgs a, double w0, double xc) {
  constexpr int N = C::N;
  extern __shared__ float4 smem_f4[];
  float2* s_twf = reinterpret_cast<float2*>(smem_f4);
  float2* s_twi = s_twf + C::TWF;
  float2* s_buf = s_twi + C::TWI + C::TW4;
  float2* line = s_buf + C::BUFLEN;
  __shared__ double s_part[kThreads];
  load_twiddles(a.tw, s_twf, cfg_twiddles<C>());
  const double nd = __dmul_rn((double)N, a.dx);
  // sum of A(kx) over propagating bins (FP64)
  double part = 0.0;
  for (int x = threadIdx.x; x < N; x += kThreads) {
    const int f = x < (N + 1) / 2 ? x : x - N;
    const double kx = __ddiv_rn(__dmul_rn(6.283185307179586, (double)f), nd);
    const double kz2 = __dsub_rn(__dmul_rn(a.k0n0, a.k0n0), __dmul_rn(kx, kx));
    if (kz2 > 0.0) {
      const double u = kx * w0 * 0.5;
      part += exp(-u * u);
    }
  }
  s_part[threadIdx.x] = part;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) s_part[threadIdx.x] += s_part[threadIdx.x + s];
    __syncthreads();
  }
  const double sumA = s_part[0];
  for (int x = threadIdx.x; x < N; x += kThreads) {
    const int f = x < (N + 1) / 2 ? x : x - N;
    const double kx = __ddiv_rn(__dmul_rn(6.283185307179586, (double)f), nd);
    const double kz2 = __dsub_rn(__dmul_rn(a.k0n0, a.k0n0), __dmul_rn(kx, kx));
    float2 sv = make_float2(0.f, 0.f);
    if (kz2 > 0.0) {
      const double u = kx * w0 * 0.5;
      const double amp = exp(-u * u) / sumA;
      double ph = -(kx * xc) - sqrt(kz2) * a.zf;
      ph -= 6.283185307179586 * rint(ph * 0.15915494309189535);
      double sn, cs;
      sincos(ph, &sn, &cs);
      sv = make_float2((float)(amp * cs), (float)(amp * sn));
    }
    line[C::f(x)] = sv;
  }
  __syncthreads();
  // the first warp (or the first group when a group spans several warps):
  // all of its groups transform the line, group 0 writes it back
  constexpr int LT = C::T > 32 ? C::T : 32;
  if (threadIdx.x < LT) {
    const int t = C::lane();
    const int g = C::group();
    float2 v[C::PTS];
#pragma unroll
    for (int q = 0; q < C::PTS; ++q) v[q] = line[C::f(layout_index<N, C::T, C::RL>(q, t))];
    group_sync<C::T>(C::bar(g));
    C::inv(v, s_buf + g * C::GS, s_twf, s_twi, t, C::bar(g));
    if (g == 0) {
#pragma unroll
      for (int q = 0; q < C::PTS; ++q) line[C::f(layout_index<N, C::T, C::R0>(q, t))] = v[q];
    }
  }
  __syncthreads();
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < (size_t)N * a.ny;
       i += (size_t)gridDim.x * kThreads) {
    const int x = (int)(i % N);
    __stcg(a.work + i, line[C::f(x)]);
  }
}

// ---------------------------------------------------------------------------
// batched propagation: many independent square instances, one persistent launch
// ---------------------------------------------------------------------------
// Every thread-block cluster is a team: it takes the next instance from a
// device work queue (instances are queued largest first), runs all of that
// instance's slices, its CTAs handing the field to each other through L2
// (by the tagged exchange of the persistent kernel for small sizes, the
// cluster's CTAs being resident together, else with the cluster's hardware
// barrier between half-steps, release/acquire at cluster scope), then takes
// the next one.  No grid-wide
// barrier is involved, so clusters run independently and instances of
// different sizes mix freely.

// One queue position for a team (its leader thread): the main launch takes
// positions from the front of the order, a fill launch of smaller teams (on
// the SMs the main clusters leave free) from the back; one 64-bit word holds
// both counts, so the two ends never hand out the same position.  Returns
// n_inst when nothing is left for this taker.  Lock-free: a failed exchange
// means another team took a position; bounded all the same.
__device__ __forceinline__ int batch_take(const BatchArgs& b) {
  for (int tries = 0; tries < (1 << 20); ++tries) {
    const unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(b.queue);
    const unsigned front = (unsigned)(cur >> 32), back = (unsigned)cur;
    if (front + back >= (unsigned)b.n_inst) return b.n_inst;
    int k;
    unsigned long long next;
    if (!b.from_back) {
      k = (int)front;
      next = cur + (1ull << 32);
    } else {
      k = b.n_inst - 1 - (int)back;
      if (k < b.back_min) return b.n_inst;
      next = cur + 1ull;
    }
    if (atomicCAS(b.queue, cur, next) == cur) return k;
  }
  atomicCAS(b.err, 0, kDevErrTimeout);
  return b.n_inst;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}

template <class C>
__device__ __forceinline__ void batch_instance(const InstArgs& ia, const BatchArgs& b, int rank, int CL,
                                               float2* smem, bool& bad) {
  constexpr int N = C::N;
  float2* s_twf = smem;
  float2* s_twi = s_twf + C::TWF;
  float2* s_buf = s_twi + C::TWI + C::TW4;
  StepArgs a = {};          // every field not set below is zero / nullptr (e.g. no adapted expansion)
  a.work = ia.work;
  a.ein = ia.ein;
  a.dn = ia.dn;
  a.inten = ia.inten;
  a.iz0 = ia.iz0;
  a.iz1 = ia.iz1;
  a.nx = N;
  a.ny = N;
  a.ht = ia.ht;
  a.tw = ia.tw;
  a.screen_c = ia.screen_c;
  a.carrier = ia.carrier;
  a.z_begin = ia.z_begin;
  a.z_end = ia.z_end;
  a.err = b.err;
  a.timeout_ns = b.timeout_ns;
  a.tag_stall = b.tag_stall;
  a.accumulate = 0;
  a.out = nullptr;
  const int lo = (rank * N) / CL, hi = ((rank + 1) * N) / CL;
  if (a.z_end <= a.z_begin) {
    // empty slice range: the output is the input
    if (a.work != a.ein)
      for (int i = lo * N + threadIdx.x; i < hi * N; i += kThreads) __stcg(a.work + i, __ldcg(a.ein + i));
    cluster_sync_all();
    return;
  }
  load_twiddles(a.tw, s_twf, cfg_twiddles<C>());
  // Small sizes hand the field between their half-steps through tagged
  // elements (as the persistent kernel does): the cluster barrier after the
  // entrance field's forward FFT_x makes its tagged writes visible, a CTA
  // barrier separates the half-steps' uses of shared memory, and a failed
  // wait ends the instance for this CTA (the others' waits give up on the
  // error word).  Their slices are short (a 128^2 slice on 8 CTAs: 7.5 ->
  // 6.4 us).  From 256 on, each CTA takes several rounds of rows or columns
  // per half-step and the cluster's hardware barrier costs less than the
  // polls (512^2: 54 us with the barrier, 58 us tagged).
  constexpr bool TGB = N <= 192;
  row_half_step<C, N, ROW_FWD, false, true, TGB>(a, lo, hi, a.z_begin, s_buf, s_twf, s_twi, bad);
  cluster_sync_all();
  for (int z = a.z_begin; z < a.z_end; ++z) {
    bool ok = col_half_step<C, N, COL_PROP, 0, TGB>(a, lo, hi, z, s_buf, s_twf, s_twi);
    if constexpr (TGB) {
      if (__syncthreads_or(!ok)) break;
    } else {
      cluster_sync_all();
    }
    if (z + 1 < a.z_end) ok = row_half_step<C, N, ROW_STEP, false, false, TGB>(a, lo, hi, z, s_buf, s_twf, s_twi, bad);
    else ok = row_half_step<C, N, ROW_LAST, false, false, TGB>(a, lo, hi, z, s_buf, s_twf, s_twi, bad);
    if constexpr (TGB) {
      if (__syncthreads_or(!ok)) break;
    } else {
      cluster_sync_all();
    }
  }
}

}  // namespace bpmk
