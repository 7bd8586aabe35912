// bpm_args.cuh - argument blocks shared by the host side (bpm.cu) and the
// device code of the split-step beam-propagation library.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace bpmk {

constexpr int kThreads = 256;   // CTA size for every kernel of the path
constexpr int kWarps = kThreads / 32;

// device error codes (match the negative BPM_ERR_* values of bpm.h)
constexpr int kDevErrTimeout = -4;
constexpr int kDevErrNan = -5;

// What a half-step launch does: rows (forward transform of the entrance
// field; one propagation step's row half; the last slice's; inverse transform
// accumulated into an output) or columns (propagator; focusing filter of the
// multiplexed synthesis).
enum RowMode { ROW_FWD = 0, ROW_STEP = 1, ROW_LAST = 2, ROW_INV_ACC = 3 };
enum ColMode { COL_PROP = 0, COL_FOCUS = 1 };

// Everything one propagation (or synthesis) launch needs.  The field is
// [ny][nx] row-major: rows have length nx, columns length ny.
struct StepArgs {
  float2* work;            // [ny][nx] working field; holds E_out at the end
  const float2* ein;       // [ny][nx] input field (read once)
  const __half* dn;        // [nz][ny][nx] index volume (dn = n - n0)
  float* inten;            // [iz1 - iz0][ny][nx] or nullptr
  int iz0, iz1;            // intensity window: slice z in [iz0, iz1) goes to inten[z - iz0]
  int nx, ny;              // grid (row length, column length)
  // per-half-step launches of a grid whose row and column transforms differ
  // in kind (rolled loop or not): the column kernel conjugates its output
  // so that the row kernel receives the hand-off it expects
  int flip_col;
  // locally adapted expansion (reading B), nullptr when off: the mean index
  // step of each slice and G = k0^2 n0 dz / kz0 per component, transposed
  // like ht; slice z's propagator is H exp(i delta[z] G), its screen acts on
  // dn - delta[z]
  const float* delta;
  const float* gt;
  // propagation towards -z: loop step z handles slice z_begin + z_end - 1 - z
  // (index, slice mean and intensity of that slice); the field enters at the
  // exit plane of slice z_end - 1
  int reverse;
  // complex index (absorption): imaginary part kappa of n per voxel,
  // [nz][ny][nx] FP16, or nullptr; the screen attenuates by exp(-k0 kappa dz)
  const __half* kappa;
  const float2* ht;        // [nx][ny] propagator, transposed: ht[kx * ny + ky]
  const float2* tw;        // twiddles of the launch's transforms (row tables, then column tables)
  float screen_c;          // k0 dz
  float2 carrier;          // exp(i k0 n0 dz (z_end - z_begin))
  int z_begin, z_end;
  // focusing filter (synthesis): multiplier exp(-i kz zf) / (nx ny) inside the pupil
  double k0n0, kna2, zf, dx, dy;   // k0 n0, (k0 NA)^2, focal depth, lateral spacings
  double kin2;                     // (k0 NA_in)^2: inner edge of an annular pupil (0 for a disk)
  int accumulate;                  // INV_ACC: add into out instead of storing
  float2* out;                     // INV_ACC destination
  // team barrier
  unsigned* bar;
  int* err;
  unsigned long long timeout_ns;
  unsigned bar_extra;
  // test hook: the entrance field's forward transform writes the tag the row
  // half-steps write (1 instead of 0), so the first tagged wait runs out
  int tag_stall;
  // persistent kernel: rows and columns per CTA at most, and which per-CTA
  // buffers live in shared memory (propagator columns, index rows)
  int rmax_r, rmax_c;
  int h_res, dn_stage;
};

// batched propagation (square grids): one instance's arguments
struct InstArgs {
  float2* work;
  const float2* ein;
  const __half* dn;
  float* inten;
  const float2* ht;
  const float2* tw;
  float screen_c;
  float2 carrier;
  int n, z_begin, z_end;
  int iz0, iz1;             // intensity window (as in StepArgs)
};

struct BatchArgs {
  const InstArgs* inst;         // [n_inst]
  const int* order;             // queue order (instance indices, largest first)
  int n_inst;
  unsigned long long* queue;    // (taken from the front << 32) | taken from the back, zeroed before the launch
  int* slots;                   // per-cluster broadcast of the fetched queue position
  int slot_base;                // this launch's first slot (a fill launch follows the main one)
  int from_back;                // 0: take from the front (largest first); 1: from the back (smallest first)
  int back_min;                 // a back taker takes no position below this (too large for its team)
  int* err;
  unsigned long long timeout_ns;  // limit of every device wait (tagged exchange, queue)
  int tag_stall;                  // test hook, as StepArgs::tag_stall (tagged instance sizes)
};

// Position of the twiddle of butterfly b, radix element r, thread t within
// one pass's table of a transform with T threads: [b][r][t], or with `paired`
// (rolled-loop transforms, even R) [b][r/2][t][r%2] so that a thread reads
// the twiddles of r and r + 1 with one 16-byte load.  The host and device
// table builders both use it, so their layouts cannot drift apart.
__host__ __device__ inline size_t twiddle_slot(int b, int r, int t, int R, int T, bool paired) {
  return paired ? ((size_t)(b * (R / 2) + r / 2) * T + t) * 2 + (r & 1) : (size_t)(b * R + r) * T + t;
}

// Rounding of a unit-modulus twiddle (c, s) = (cos, sin) to FP32.  The
// transforms apply the same twiddles in every slice, so their rounding errors
// add up coherently over the depth, and the modulus error |w|^2 - 1 is the
// part that does not cancel between a transform and its inverse.  Of the 3 x 3
// pairs one ulp around the round-to-nearest pair, this takes the one whose
// squared modulus (in FP64) is closest to 1, ties to the nearer pair: the
// modulus error falls from 3.3e-8 to 2.2e-8 rms over the 1024-point
// twiddles, and the field error of 1024 homogeneous 1024^2 slices from
// 1.58e-4 to 1.14e-4 (a wider search trades too much angle for modulus and
// was worse: 1.98e-4 at two ulps).
__host__ __device__ inline float ulp_step(float x, int dir) {
  if (dir == 0) return x;
#ifdef __CUDA_ARCH__
  return nextafterf(x, dir > 0 ? 1e30f : -1e30f);
#else
  return std::nextafter(x, dir > 0 ? 1e30f : -1e30f);
#endif
}
__host__ __device__ inline float2 round_unit(double c, double s) {
  const float c0 = (float)c, s0 = (float)s;
  float2 best = make_float2(c0, s0);
  double bm = 1e300, bd = 1e300;
  for (int i = -1; i <= 1; ++i)
    for (int j = -1; j <= 1; ++j) {
      const float cc = ulp_step(c0, i), ss = ulp_step(s0, j);
      const double m = (double)cc * cc + (double)ss * ss - 1.0;
      const double am = m < 0 ? -m : m;
      const double d = ((double)cc - c) * ((double)cc - c) + ((double)ss - s) * ((double)ss - s);
      if (am < bm || (am == bm && d < bd)) {
        bm = am;
        bd = d;
        best = make_float2(cc, ss);
      }
    }
  return best;
}

}  // namespace bpmk
