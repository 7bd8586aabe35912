// fft.cuh - register/shared-memory FFT building blocks for sm_103a.
//
// One 1D transform of length N is computed by a group of T threads (a part of
// one warp, synchronised by __syncwarp, or whole warps, synchronised by a
// named barrier of the group).  Each thread
// keeps N/T points in registers.  The transform is a mixed-radix Stockham
// decomposition N = R_0 R_1 ... R_{P-1}: pass p performs N/R_p radix-R_p
// butterflies (B = N/(R_p T) per thread) fully in registers, and the passes
// exchange data through a per-group shared-memory buffer.  The Stockham order
// keeps the output in natural order without a bit-reversal step:
//
//   pass p (Ns = R_0 ... R_{p-1}), butterfly j in [0, N/R_p):
//     inputs  x[j + r N/R_p], r < R_p
//     twiddle x_r *= W_{Ns R_p}^{(j mod Ns) r}
//     R_p-point DFT in registers
//     outputs y[(j / Ns) Ns R_p + (j mod Ns) + r Ns]
//
// Register layout L(R): thread t holds, in v[b R + r], the element
// j + r N/R with j = t + b T.  A transform with radices (R_0..R_{P-1}) reads
// L(R_0) and leaves L(R_{P-1}) in registers; running the inverse with the
// radices reversed therefore consumes the forward output in place, and the
// pointwise propagator/screen multiplies between transforms never touch
// shared memory.
//
// Twiddles between passes come from a per-thread table in shared memory
// (laid out [pass][b][r][t], so reads are bank-conflict free), built in FP64
// on the host and rounded once to float (round_unit).  Constant twiddles
// inside the register DFTs are compile-time values of cos/sin evaluated by a
// constexpr Taylor series and rounded the same way (ct_unit).
#pragma once
#include <cuda_runtime.h>
#include <utility>

namespace bpmk {

// ---------------------------------------------------------------------------
// compile-time trigonometry (Taylor series, evaluated by the compiler only)
// ---------------------------------------------------------------------------
constexpr double kPiD = 3.14159265358979323846264338327950288;

__host__ __device__ constexpr double ct_sin(double x) {
  // x in [-pi, pi]; 30 terms leave a truncation error far below 1e-20.
  double term = x, sum = x;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double ct_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
// angle 2 pi e / R reduced to (-pi, pi]
__host__ __device__ constexpr double ct_angle(int e, int R) {
  int m = ((e % R) + R) % R;
  double a = 2.0 * kPiD * (double)m / (double)R;
  return a > kPiD ? a - 2.0 * kPiD : a;
}

// Compile-time counterpart of round_unit (bpm_args.cuh) for the constant
// twiddles inside the register DFTs: one ulp of a normal float, and the pair
// one ulp around the rounded (c, s) whose squared modulus is closest to 1.
__host__ __device__ constexpr double ct_ulp(float x) {
  double a = x < 0 ? -(double)x : (double)x;
  if (a == 0.0) return 1.401298464324817e-45;
  double p = 1.0;
  while (p > a) p *= 0.5;
  while (p * 2.0 <= a) p *= 2.0;
  return p / 8388608.0;   // 2^-23 of the binade of x
}
struct CtPair {
  float c, s;
};
__host__ __device__ constexpr CtPair ct_unit(double c, double s) {
  const float c0 = (float)c, s0 = (float)s;
  CtPair best{c0, s0};
  double bm = 1e300, bd = 1e300;
  for (int i = -1; i <= 1; ++i)
    for (int j = -1; j <= 1; ++j) {
      const float cc = (float)((double)c0 + i * ct_ulp(c0)), ss = (float)((double)s0 + j * ct_ulp(s0));
      const double m = (double)cc * cc + (double)ss * ss - 1.0;
      const double am = m < 0 ? -m : m;
      const double d = ((double)cc - c) * ((double)cc - c) + ((double)ss - s) * ((double)ss - s);
      if (am < bm || (am == bm && d < bd)) {
        bm = am;
        bd = d;
        best = CtPair{cc, ss};
      }
    }
  return best;
}

template <int... Is, class F>
__device__ __forceinline__ void static_for_impl(std::integer_sequence<int, Is...>, F&& f) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(std::make_integer_sequence<int, N>{}, f);
}
// f(q) for q = 0 .. NQ - 1: unrolled (U; q a compile-time value in each copy)
// or one rolled loop (a single copy of the body, q at run time)
template <bool U, int NQ, class F>
__device__ __forceinline__ void pass_loop(F&& f) {
  if constexpr (U) {
    static_for<NQ>([&](auto q) { f(decltype(q)::value); });
  } else {
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) f(q);
  }
}

// ---------------------------------------------------------------------------
// complex helpers (float2 = re, im)
// ---------------------------------------------------------------------------
// Sums and differences use the packed two-lane FP32 add of sm_100 and later
// (one instruction per complex value, rounding identical to two scalar adds);
// the transforms are issue-bound, so this takes 1.5-3.5 % off a slice.  The
// products stay scalar: forming the broadcast operand pairs of a packed
// complex product costs more moves than it saves.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a b) and conj(a) b: the conjugations of an inverse transform taken as
// a conjugated forward one, folded into a neighbouring product (negations
// are free operand modifiers of the scalar products)
__device__ __forceinline__ float2 cmul_conj_out(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(-a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cmul_conj_in(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
// multiply by S*i (S = +-1)
template <int S>
__device__ __forceinline__ float2 mul_si(float2 a) {
  return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// a * W_R^E with W_R = exp(S 2 pi i / R); E, R compile-time
template <int E, int R, int S>
__device__ __forceinline__ float2 twc(float2 a) {
  constexpr int e = ((E % R) + R) % R;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (4 * e == R) {
    return mul_si<S>(a);
  } else if constexpr (2 * e == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * e == 3 * R) {
    return mul_si<-S>(a);
  } else {
    constexpr CtPair w = ct_unit(ct_cos(ct_angle(e, R)), S * ct_sin(ct_angle(e, R)));
    return cmul(a, make_float2(w.c, w.s));
  }
}

// Synchronise the T threads of one transform group: a warp-level barrier
// when the group sits inside one warp, else the named CTA barrier bar_id
// (1..15) over the group's T threads (T a multiple of 32).
template <int T>
__device__ __forceinline__ void group_sync(int bar_id) {
  if constexpr (T <= 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "n"(T) : "memory");
  }
}

// ---------------------------------------------------------------------------
// R-point DFT in registers, natural order in and out, sign S
// ---------------------------------------------------------------------------
template <int R, int S>
struct Dft;

template <int S>
struct Dft<1, S> {
  __device__ __forceinline__ static void run(float2*) {}
};
template <int S>
struct Dft<2, S> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};
template <int S>
struct Dft<3, S> {
  __device__ __forceinline__ static void run(float2* v) {
    constexpr float h = (float)(S * 0.86602540378443864676372317075294);  // S sqrt(3)/2
    float2 a = v[0], b = v[1], c = v[2];
    float2 t1 = cadd(b, c);
    float2 t2 = make_float2(fmaf(-0.5f, t1.x, a.x), fmaf(-0.5f, t1.y, a.y));
    float2 d = csub(b, c);
    float2 t3 = make_float2(-h * d.y, h * d.x);  // i S sqrt(3)/2 (b - c)
    v[0] = cadd(a, t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
  }
};
template <int S>
struct Dft<4, S> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a = v[0], b = v[1], c = v[2], d = v[3];
    float2 s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(b, d), s3 = mul_si<S>(csub(b, d));
    v[0] = cadd(s0, s2);
    v[2] = csub(s0, s2);
    v[1] = cadd(s1, s3);
    v[3] = csub(s1, s3);
  }
};

// composite R = P M, decimation in time:
//   X[k1 + M k2] = DFT_P over n1 of ( W_R^{n1 k1} DFT_M over n2 of x[P n2 + n1] )
template <int R, int S>
struct Dft {
  static constexpr int P = (R % 4 == 0) ? 4 : ((R % 2 == 0) ? 2 : 3);
  static constexpr int M = R / P;
  static_assert(P * M == R && M > 1, "radix must be a product of 2s and 3s");
  __device__ __forceinline__ static void run(float2* v) {
    float2 u[P][M];
    static_for<P>([&](auto I1) {
      constexpr int n1 = decltype(I1)::value;
      static_for<M>([&](auto I2) {
        constexpr int n2 = decltype(I2)::value;
        u[n1][n2] = v[P * n2 + n1];
      });
      Dft<M, S>::run(u[n1]);
      static_for<M>([&](auto K1) {
        constexpr int k1 = decltype(K1)::value;
        u[n1][k1] = twc<n1 * k1, R, S>(u[n1][k1]);
      });
    });
    static_for<M>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      float2 w[P];
      static_for<P>([&](auto I1) { w[decltype(I1)::value] = u[decltype(I1)::value][k1]; });
      Dft<P, S>::run(w);
      static_for<P>([&](auto K2) {
        constexpr int k2 = decltype(K2)::value;
        v[k1 + M * k2] = w[k2];
      });
    });
  }
};

// Order in which Dft<R> first consumes its inputs and last produces its
// outputs: inputs by decimation subsequence (n1 + P n2, n1 outer), outputs by
// final P-point DFT (k1 + M k2, k1 outer).  Loads issued in the first order
// let the first inner DFTs start while later loads are still in flight;
// stores issued in the second follow the values as they are finished.
template <int R>
__host__ __device__ constexpr int dft_input_order(int i) {
  constexpr int P = (R % 4 == 0) ? 4 : ((R % 2 == 0) ? 2 : 3);
  constexpr int M = R / P;
  return (R <= 4 || P * M != R) ? i : P * (i % M) + i / M;
}
template <int R>
__host__ __device__ constexpr int dft_output_order(int i) {
  constexpr int P = (R % 4 == 0) ? 4 : ((R % 2 == 0) ? 2 : 3);
  constexpr int M = R / P;
  return (R <= 4 || P * M != R) ? i : i / P + M * (i % P);
}

// ---------------------------------------------------------------------------
// group transform over shared memory (mixed radices, fully unrolled)
// ---------------------------------------------------------------------------
template <int... Rs>
struct Radices {
  static constexpr int count = sizeof...(Rs);
  __host__ __device__ static constexpr int at(int i) {
    constexpr int vals[] = {Rs...};
    return vals[i];
  }
  __host__ __device__ static constexpr int product() {
    int p = 1;
    for (int i = 0; i < count; ++i) p *= at(i);
    return p;
  }
  __host__ __device__ static constexpr int prefix(int p) {
    int q = 1;
    for (int i = 0; i < p; ++i) q *= at(i);
    return q;
  }
};

// N points, T threads per group, shared-memory index padding one slot every
// PAD elements, sign S (-1 forward, +1 inverse), radix list RS.
template <int N_, int T_, int PAD_, int S_, class RS>
struct GroupFFT {
  static constexpr int N = N_, T = T_, PAD = PAD_, S = S_;
  using Rad = RS;
  static constexpr int NP = RS::count;
  static constexpr int PTS = N / T;
  static constexpr int R0 = RS::at(0);
  static constexpr int RL = RS::at(NP - 1);
  static constexpr int BUF = N + N / PAD;          // exchange buffer length (float2)
  static constexpr int TW = (NP - 1) * N;          // twiddle table length (float2)
  static_assert(RS::product() == N, "radices must multiply to N");
  static_assert((T <= 32 && 32 % T == 0) || T % 32 == 0, "a group is part of one warp or whole warps");

  __device__ __forceinline__ static int f(int i) { return i + i / PAD; }

  template <int p>
  __device__ __forceinline__ static void pass(float2* v, float2* buf, const float2* tw, int t, int bar_id) {
    constexpr int R = RS::at(p);
    constexpr int B = N / (R * T);
    constexpr int Ns = RS::prefix(p);
    static_assert(B * R * T == N, "each thread must own whole butterflies");
    if constexpr (p > 0) {
      const float2* twp = tw + (p - 1) * N;
#pragma unroll
      for (int b = 0; b < B; ++b)
#pragma unroll
        for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], twp[(b * R + r) * T + t]);
    }
#pragma unroll
    for (int b = 0; b < B; ++b) Dft<R, S>::run(v + b * R);
    if constexpr (p + 1 < NP) {
#pragma unroll
      for (int b = 0; b < B; ++b) {
        int j = t + b * T;
        int jm = j % Ns;
        int base = (j / Ns) * Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[f(base + r * Ns)] = v[b * R + r];
      }
      group_sync<T>(bar_id);
      constexpr int Rn = RS::at(p + 1);
      constexpr int Bn = N / (Rn * T);
#pragma unroll
      for (int b = 0; b < Bn; ++b) {
        int j = t + b * T;
#pragma unroll
        for (int r = 0; r < Rn; ++r) v[b * Rn + r] = buf[f(j + r * (N / Rn))];
      }
      group_sync<T>(bar_id);
      pass<p + 1>(v, buf, tw, t, bar_id);
    }
  }

  // v: L(R0) in, L(RL) out.  buf: this group's BUF-long exchange buffer.
  // tw: this transform's twiddle table (TW entries, may be in shared memory).
  // bar_id: named barrier of the group when T > 32 (unused otherwise).
  __device__ __forceinline__ static void run(float2* v, float2* buf, const float2* tw, int t, int bar_id = 0) {
    pass<0>(v, buf, tw, t, bar_id);
  }
};

// ---------------------------------------------------------------------------
// uniform-radix transform with a rolled pass loop
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ilog2_ceil(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}
__host__ __device__ constexpr int ilog_ceil(int n, int r) {
  int p = 0;
  long long q = 1;
  while (q < n) {
    q *= r;
    ++p;
  }
  return p;
}

__device__ __forceinline__ void conj_all(float2* v, int n) {
#pragma unroll
  for (int k = 0; k < n; ++k) v[k].y = -v[k].y;
}

// N = R^NP with R a power of two.  The same Stockham passes as GroupFFT, one
// pass function for every pass of both directions: the inverse transform is
// computed as conj(DFT(conj(x))) with the forward twiddles.  With U false the
// pass index is a runtime loop variable, so one copy of the radix-R code
// serves all passes and the instruction footprint of a half-step stays a few
// KiB (for kernels whose one instruction stream holds several sizes); with U
// true the passes are unrolled, so that the pass index, the twiddle addresses
// and the exchange branches are compile-time (every configuration uses this:
// 6-13 % shorter slices than the rolled loop).
template <int N_, int T_, int R_, int PAD_, bool U_ = false>
struct LoopFFT {
  static constexpr int N = N_, T = T_, R = R_, PAD = PAD_;
  static constexpr int R0 = R_, RL = R_;
  static constexpr int NP = ilog_ceil(N_, R_);
  static constexpr int LGR = ilog2_ceil(R_);
  static constexpr int PTS = N / T;
  static constexpr int B = N / (R * T);
  static constexpr int BUF = N + N / PAD;
  static constexpr int TW = (NP - 1) * N;
  static_assert((1 << LGR) == R && R >= 2, "radix must be a power of two (even: paired twiddles)");
  static_assert(B * R * T == N && B >= 1, "each thread must own whole butterflies");
  static_assert((T <= 32 && 32 % T == 0) || T % 32 == 0, "a group is part of one warp or whole warps");

  __device__ __forceinline__ static int f(int i) { return i + i / PAD; }

  // forward Stockham pass p; registers L(R) in and out
  __device__ __forceinline__ static void pass(int p, float2* v, float2* buf, const float2* tw, int t,
                                              int bar_id = 0) {
    if (p > 0) {
      // table [pass][b][r/2][t][r%2]: the twiddles of r and r + 1 in one
      // 16-byte load (the table starts 16-byte aligned)
      const float4* twp = reinterpret_cast<const float4*>(tw + (p - 1) * N);
#pragma unroll
      for (int b = 0; b < B; ++b)
#pragma unroll
        for (int rp = 0; rp < R / 2; ++rp) {
          const float4 w = twp[(b * (R / 2) + rp) * T + t];
          if (rp > 0) v[b * R + 2 * rp] = cmul(v[b * R + 2 * rp], make_float2(w.x, w.y));
          v[b * R + 2 * rp + 1] = cmul(v[b * R + 2 * rp + 1], make_float2(w.z, w.w));
        }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) Dft<R, -1>::run(v + b * R);
    if (p + 1 < NP) {
      // Ns = R^p = 1 << lg; with two passes only pass 0 exchanges, so the
      // store addresses are compile-time offsets from the thread's base
      const int lg = NP == 2 ? 0 : p * LGR;
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int j = t + b * T;
        const int base = ((j >> lg) << (lg + LGR)) + (j & ((1 << lg) - 1));
#pragma unroll
        for (int r = 0; r < R; ++r) buf[f(base + (r << lg))] = v[b * R + r];
      }
      group_sync<T>(bar_id);
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int j = t + b * T;
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = buf[f(j + r * (N / R))];
      }
      group_sync<T>(bar_id);
    }
  }

  __device__ __forceinline__ static void run_fwd(float2* v, float2* buf, const float2* tw, int t, int bar_id = 0) {
    pass_loop<U_, NP>([&](int p) { pass(p, v, buf, tw, t, bar_id); });
  }
  __device__ __forceinline__ static void run_inv(float2* v, float2* buf, const float2* tw, int t, int bar_id = 0) {
    conj_all(v, PTS);
    pass_loop<U_, NP>([&](int p) { pass(p, v, buf, tw, t, bar_id); });
    conj_all(v, PTS);
  }
};

// element index held in v[k] under layout L(R) for thread t
template <int N, int T, int R>
__device__ __forceinline__ int layout_index(int k, int t) {
  return (t + (k / R) * T) + (k % R) * (N / R);
}

}  // namespace bpmk
