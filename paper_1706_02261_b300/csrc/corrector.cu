// corrector.cu - learned coarse-step corrector: training and inference kernels.
//
// A 4-layer 3x3 convolutional network (C_in -> 32 -> 32 -> 32 -> 2, ReLU
// between, circular padding, residual output out = x[:, :2] + f(x)) corrects
// the field after each coarse split-step of length 4 dz.  Weights are kept as
// FP32 masters with Adam moments; the convolutions use the BF16-rounded
// weights (stored as float) and accumulate in FP32.  Layout of every activation
// tensor: [batch][channel][y][x] float; H and W multiples of 16.
//
// Training kernels on the FP32 pipes (direct convolutions; the tensor-core
// training path of bpm_corrector_set_train_tensor_cores is in namespace tc):
//   corr_conv      forward conv (+bias, +ReLU) and, with TRANS, the adjoint
//                  (transposed) conv of backpropagation with the ReLU mask of
//                  the layer below fused in; one 16x16 output tile per CTA, the
//                  input tile with a 1-pixel circular halo and the layer's
//                  weights in shared memory, weights read 4 output channels at
//                  a time.
//   corr_wgrad     per-tile partial weight and bias gradients (each thread:
//                  one input channel x 4 output channels x 9 taps), then
//   corr_reduce    a deterministic sum of the partials over tiles.
//   corr_loss      residual output, squared error and d loss / d Z4.
//   corr_adam      Adam update of the masters and the BF16 working copy.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bpm.h"
#include "bpm_corrector.h"

namespace {

constexpr int kCh = 32;          // hidden channels
constexpr int kTile = 16;        // output tile edge
constexpr int kHalo = kTile + 2;
constexpr int kTilePix = kHalo * kHalo;

thread_local std::string g_corr_err;
int cfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_corr_err = buf;
  return code;
}
#define CORR_CU(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return cfail(BPM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// out[b][co][p] = sum_{ci, tap} w(co, ci, tap) in[b][ci][p + off(tap)] (+ bias)
//   forward : w(co, ci, tap) = W[co][ci][tap]            (layer CIN -> COUT)
//   TRANS   : w(co, ci, tap) = W[ci][co][8 - tap]        (adjoint of a COUT <- CIN layer)
// MASK multiplies by (mask > 0) (ReLU derivative of the layer below); RELU also
// stores max(out, 0).
template <int CIN, int COUT, bool TRANS, bool BIAS, bool MASK, bool RELU>
__global__ void __launch_bounds__(256) corr_conv(const float* __restrict__ in, const float* __restrict__ Wt,
                                                 const float* __restrict__ bias, const float* __restrict__ mask,
                                                 float* __restrict__ Z, float* __restrict__ A, int H, int W) {
  extern __shared__ float4 sm4[];
  float* tile = reinterpret_cast<float*>(sm4);              // [CIN][18*18]
  float* wsm = tile + ((CIN * kTilePix + 3) & ~3);          // [CIN][9][COUT]
  const int b = blockIdx.z, y0 = blockIdx.y * kTile, x0 = blockIdx.x * kTile;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < CIN * kTilePix; idx += 256) {
    const int ci = idx / kTilePix, r = idx % kTilePix;
    const int gy = (y0 + r / kHalo - 1 + H) % H, gx = (x0 + r % kHalo - 1 + W) % W;
    tile[idx] = in[(((size_t)b * CIN + ci) * H + gy) * W + gx];
  }
  for (int idx = tid; idx < CIN * 9 * COUT; idx += 256) {
    const int co = idx % COUT, rem = idx / COUT, tap = rem % 9, ci = rem / 9;
    wsm[idx] = TRANS ? Wt[(ci * COUT + co) * 9 + (8 - tap)] : Wt[(co * CIN + ci) * 9 + tap];
  }
  __syncthreads();
  const int ty = tid / kTile, tx = tid % kTile;
  float acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = BIAS ? bias[co] : 0.f;
  for (int ci = 0; ci < CIN; ++ci) {
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const float v = tile[ci * kTilePix + (ty + tap / 3) * kHalo + tx + tap % 3];
      const float* wr = wsm + (ci * 9 + tap) * COUT;
      if constexpr (COUT % 4 == 0) {
#pragma unroll
        for (int co = 0; co < COUT; co += 4) {
          const float4 w4 = *reinterpret_cast<const float4*>(wr + co);
          acc[co] = fmaf(w4.x, v, acc[co]);
          acc[co + 1] = fmaf(w4.y, v, acc[co + 1]);
          acc[co + 2] = fmaf(w4.z, v, acc[co + 2]);
          acc[co + 3] = fmaf(w4.w, v, acc[co + 3]);
        }
      } else {
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = fmaf(wr[co], v, acc[co]);
      }
    }
  }
  const int y = y0 + ty, x = x0 + tx;
#pragma unroll
  for (int co = 0; co < COUT; ++co) {
    const size_t o = (((size_t)b * COUT + co) * H + y) * W + x;
    float out = acc[co];
    if constexpr (MASK) out = mask[o] > 0.f ? out : 0.f;
    Z[o] = out;
    if constexpr (RELU) A[o] = fmaxf(out, 0.f);
  }
}

template <int CIN, int COUT>
constexpr size_t conv_smem() {
  return sizeof(float) * (((CIN * kTilePix + 3) & ~3) + CIN * 9 * COUT);
}

// Partial gradients of one 16x16 tile: dW[co][ci][tap] = sum_p dZ[co][p] X[ci][p + off(tap)],
// db[co] = sum_p dZ[co][p]; written to partial[tile][P], P = COUT*CIN*9 + COUT.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) corr_wgrad(const float* __restrict__ X, const float* __restrict__ dZ,
                                                  float* __restrict__ partial, int H, int W) {
  constexpr int CG = COUT < 4 ? COUT : 4;        // output channels per task
  constexpr int P = COUT * CIN * 9 + COUT;
  extern __shared__ float4 sm4[];
  float* xt = reinterpret_cast<float*>(sm4);     // [CIN][18*18 + 1]
  constexpr int XS = kTilePix + 1;
  float* dzt = xt + CIN * XS;                    // [COUT][256 + 1]
  constexpr int DS = kTile * kTile + 1;
  const int b = blockIdx.z, y0 = blockIdx.y * kTile, x0 = blockIdx.x * kTile, tid = threadIdx.x;
  for (int idx = tid; idx < CIN * kTilePix; idx += 256) {
    const int ci = idx / kTilePix, r = idx % kTilePix;
    const int gy = (y0 + r / kHalo - 1 + H) % H, gx = (x0 + r % kHalo - 1 + W) % W;
    xt[ci * XS + r] = X[(((size_t)b * CIN + ci) * H + gy) * W + gx];
  }
  for (int idx = tid; idx < COUT * kTile * kTile; idx += 256) {
    const int co = idx / (kTile * kTile), p = idx % (kTile * kTile);
    dzt[co * DS + p] = dZ[(((size_t)b * COUT + co) * H + y0 + p / kTile) * W + x0 + p % kTile];
  }
  __syncthreads();
  const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  float* out = partial + blk * P;
  constexpr int TASKS = (COUT / CG) * CIN;
  for (int task = tid; task < TASKS; task += 256) {
    const int ci = task % CIN, cg = task / CIN;
    float acc[CG][9];
    float bacc[CG];
#pragma unroll
    for (int g = 0; g < CG; ++g) {
      bacc[g] = 0.f;
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[g][k] = 0.f;
    }
    for (int p = 0; p < kTile * kTile; ++p) {
      const int py = p / kTile, px = p % kTile;
      float xv[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) xv[k] = xt[ci * XS + (py + k / 3) * kHalo + px + k % 3];
#pragma unroll
      for (int g = 0; g < CG; ++g) {
        const float d = dzt[(cg * CG + g) * DS + p];
        bacc[g] += d;
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[g][k] = fmaf(d, xv[k], acc[g][k]);
      }
    }
#pragma unroll
    for (int g = 0; g < CG; ++g) {
      const int co = cg * CG + g;
#pragma unroll
      for (int k = 0; k < 9; ++k) out[(co * CIN + ci) * 9 + k] = acc[g][k];
      if (ci == 0) out[COUT * CIN * 9 + co] = bacc[g];
    }
  }
}

template <int CIN, int COUT>
constexpr size_t wgrad_smem() {
  return sizeof(float) * (CIN * (kTilePix + 1) + COUT * (kTile * kTile + 1));
}

// grad[i] = sum_t partial[t][i] (fixed order: deterministic)
__global__ void corr_reduce(const float* __restrict__ partial, int tiles, int P, float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  float s = 0.f;
  for (int t = 0; t < tiles; ++t) s += partial[(size_t)t * P + i];
  grad[i] = s;
}

// out = x[:, :2] + sigma z4; r = out - target; dz4 = 2 sigma r / n; per-block sum of r^2
__global__ void corr_loss(const float* __restrict__ x, int cin, const float* __restrict__ z4, float sigma,
                          const float* __restrict__ target, float* __restrict__ dz4, float* __restrict__ part,
                          int batch, int hw) {
  __shared__ float red[256];
  const size_t n = (size_t)batch * 2 * hw;
  float s = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / (2 * (size_t)hw), rem = i % (2 * (size_t)hw);
    const float out = fmaf(sigma, z4[i], x[b * cin * hw + rem]);
    const float r = out - target[i];
    dz4[i] = 2.f * sigma * r / (float)n;
    s = fmaf(r, r, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void corr_sum(const float* __restrict__ part, int n, float scale, float* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = (float)(red[0] * scale);
}

// out[b][:2] = x[b][:2] + sigma z4[b]
__global__ void corr_residual(const float* __restrict__ x, int cin, const float* __restrict__ z4, float sigma,
                              float* __restrict__ out, int batch, int hw) {
  const size_t n = (size_t)batch * 2 * hw;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / (2 * (size_t)hw), rem = i % (2 * (size_t)hw);
    out[i] = fmaf(sigma, z4[i], x[b * cin * hw + rem]);
  }
}

__global__ void corr_adam(float* __restrict__ master, float* __restrict__ work, float* __restrict__ m,
                          float* __restrict__ v, const float* __restrict__ g, int n, float lr, float b1, float b2,
                          float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float w = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  master[i] = w;
  work[i] = __bfloat162float(__float2bfloat16_rn(w));
}

__global__ void corr_round_bf16(const float* __restrict__ master, float* __restrict__ work, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) work[i] = __bfloat162float(__float2bfloat16_rn(master[i]));
}

// Per-field RMS amplitude a[b] = sqrt(mean |E|^2) (FP64 accumulation), one
// CTA per field; a field of zeros gets a = 1.
// RMS amplitude of each field (the normalisation the network sees; pack and
// unpack use the same value, so it needs no more than FP32 partial sums):
// kRmsChunks blocks per field sum |E|^2 over their share, then one warp per
// field combines the partials in a fixed order.
constexpr int kRmsChunks = 64;
__global__ void corr_field_rms_partial(const float2* __restrict__ field, int hw, float* __restrict__ partial) {
  __shared__ float red[256];
  const float2* f = field + (size_t)blockIdx.y * hw;
  const int per = (hw + kRmsChunks - 1) / kRmsChunks;
  const int p0 = blockIdx.x * per, p1 = min(hw, p0 + per);
  float s = 0.f;
  for (int p = p0 + threadIdx.x; p < p1; p += 256) s = fmaf(f[p].x, f[p].x, fmaf(f[p].y, f[p].y, s));
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.y * kRmsChunks + blockIdx.x] = red[0];
}
__global__ void corr_field_rms_final(const float* __restrict__ partial, int hw, float* __restrict__ amp) {
  // one warp: lane l adds partials l, l + 32, ...; then a fixed shuffle tree
  float t = 0.f;
  for (int k = threadIdx.x; k < kRmsChunks; k += 32) t += partial[blockIdx.x * kRmsChunks + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (threadIdx.x == 0) {
    const float a = sqrtf(t / (float)hw);
    amp[blockIdx.x] = a > 0.f ? a : 1.0f;
  }
}

// x[b] = [Re E / a_b, Im E / a_b, (scale * dn)] and, when target fields are
// given, t[b] = [Re T / a_b, Im T / a_b]: the network sees every field at unit
// RMS amplitude, so the correction it predicts scales linearly with the field
__global__ void corr_pack(const float2* __restrict__ field, const float2* __restrict__ tfield,
                          const __half* __restrict__ dn, float scale, const float* __restrict__ amp,
                          float* __restrict__ x, float* __restrict__ t, int cin, int batch, int hw) {
  const size_t n = (size_t)batch * hw;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / hw, p = i % hw;
    const float inv = 1.0f / amp[b];
    const float2 e = field[i];
    x[(b * cin + 0) * hw + p] = e.x * inv;
    x[(b * cin + 1) * hw + p] = e.y * inv;
    if (cin > 2) x[(b * cin + 2) * hw + p] = dn ? scale * __half2float(dn[i]) : 0.f;
    if (tfield) {
      const float2 q = tfield[i];
      t[(b * 2 + 0) * hw + p] = q.x * inv;
      t[(b * 2 + 1) * hw + p] = q.y * inv;
    }
  }
}

__global__ void corr_unpack(const float* __restrict__ out, const float* __restrict__ amp, float2* __restrict__ field,
                            int batch, int hw) {
  const size_t n = (size_t)batch * hw;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / hw, p = i % hw;
    field[i] = make_float2(out[(b * 2 + 0) * hw + p] * amp[b], out[(b * 2 + 1) * hw + p] * amp[b]);
  }
}

// out[z'][p] = FP16( mean over f of dn[z' f + k][p] ), the screen of a coarse step
__global__ void coarsen_index(const __half* __restrict__ dn, int nzc, size_t plane, int factor,
                              __half* __restrict__ out) {
  const size_t n = (size_t)nzc * plane;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t zc = i / plane, p = i % plane;
    float s = 0.f;
    for (int k = 0; k < factor; ++k) s += __half2float(dn[(zc * factor + k) * plane + p]);
    out[i] = __float2half_rn(s / (float)factor);
  }
}

int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 148 * 16); }

// ---------------------------------------------------------------------------
// Tensor-core inference path (tcgen05): each convolution as an implicit GEMM
// D[pixel][c_out] = sum over taps and c_in of A[pixel + tap][c_in] W[tap][c_in][c_out],
// BF16 operands in shared memory, FP32 accumulators in tensor memory.
//
// Activations of this path are BF16 in channel chunks of 8 with the circular
// halo stored in every row: [b][c / 8][y][W + 2][8], pixel x at column x + 1,
// column 0 repeating pixel W - 1 and column W + 1 pixel 0 (16 bytes per pixel
// and chunk), so a tile's input row with its halo is one contiguous copy, and
// the operand of a tap shifted by one pixel starts 16 bytes further: a K-major,
// unswizzled operand (core matrices of 8 pixels x 8 channels, 16 bytes per
// row) whose next 8 channels sit one chunk further (the leading byte offset)
// and whose next 8 pixels sit 128 bytes further (the stride byte offset).
// Weights: [tap][c_in / 8][c_out][8].
// ---------------------------------------------------------------------------
namespace tc {

constexpr int kM = 128;                 // output pixels per tile (one row segment)
constexpr int kPix = kM + 2;            // with the two halo pixels
constexpr int kThreadsTc = 128;         // four warps: one per quarter of the tensor-memory lanes
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// shared-memory operand descriptor: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t operand_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mbar_init(uint64_t* m) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(m)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with this parity; records a timeout in err.  The
// global timer is read only when the phase is not complete at once, and then
// every 64 polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity, int* err) {
  if (mbar_try(m, parity)) return true;
  const unsigned long long t0 = gtime();
  for (unsigned n = 1;; ++n) {
    if (mbar_try(m, parity)) return true;
    if ((n & 63) == 0 && gtime() - t0 > kWaitNs) {
      atomicCAS(err, 0, BPM_ERR_TIMEOUT);
      return false;
    }
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(m))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void commit(uint64_t* m) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(m))
               : "memory");
}
// 32 consecutive accumulator columns of this warp's 32 lanes (one pixel per thread)
__device__ __forceinline__ void ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

enum ConvOut { OUT_HIDDEN = 0, OUT_PLANES = 1, OUT_FIELD = 2, OUT_GRAD = 3 };

constexpr int kRowsTc = 2;              // output rows per tile

__host__ __device__ constexpr int tmem_cols(int n) { return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : 256)); }

// One 3x3 circular convolution layer.  CIN, COUT: channel counts padded to
// multiples of 16.  A tile is kRowsTc output rows x 128 pixels; its kRowsTc + 2
// input rows (with the two circular halo pixels) are fetched by bulk copies
// into one of two shared-memory buffers while the previous tile is computed,
// each output row's accumulators take COUT tensor-memory columns, and the
// four warps read them back (warp w: pixels 32w..32w+31).  Outputs:
//   OUT_HIDDEN  bias + ReLU, BF16 chunks [b][COUT/8][y][x][8]
//   OUT_PLANES  bias, the first cout_real channels as FP32 planes [b][c][y][x]
//   OUT_FIELD   bias, then field[b][y][x] += sigma amp[b] (f0, f1): the
//               residual update of the un-normalised field (apply)
//   OUT_GRAD    no bias; each channel times (mask > 0), mask the BF16 chunk
//               activations of the layer below: the data gradient of
//               backpropagation with the ReLU derivative (the convolution
//               then runs with the adjoint weights), BF16 chunks like OUT_HIDDEN
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(kThreadsTc) conv_tc(const __nv_bfloat16* __restrict__ in,
                                                      const __nv_bfloat16* __restrict__ wtc,
                                                      const float* __restrict__ bias, int cout_real,
                                                      __nv_bfloat16* __restrict__ out_bf, float* __restrict__ out_f,
                                                      float2* __restrict__ field, const float* __restrict__ amp,
                                                      float sigma, int B, int H, int W, int* err,
                                                      const __nv_bfloat16* __restrict__ mask = nullptr) {
  static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 32, "padded channel counts");
  static_assert(MODE != OUT_GRAD || COUT == 32, "gradients of the hidden layers (32 channels)");
  constexpr int R = kRowsTc;
  constexpr int KC = CIN / 8;
  constexpr int ROWB = KC * kPix * 16;            // one input row (all chunks) in shared memory
  constexpr int TILEB = (R + 2) * ROWB;
  constexpr int WBYTES = 9 * KC * COUT * 16;
  constexpr int NCOL = tmem_cols(R * COUT);
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char* sW = sm;
  unsigned char* const sA0 = sm + ((WBYTES + 127) & ~127);
  auto sA = [&](int buf) { return sA0 + (buf ? TILEB : 0); };
  __shared__ __align__(8) uint64_t bar_load[2], bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ float s_bias[32];
  const int tiles_x = W / kM, tiles_y = H / R, tiles = B * tiles_y * tiles_x;
  // rows y0-1 .. y0+R (circular), pixels x0-1 .. x0+128 (the stored halo), every chunk
  auto issue_load = [&](int tile, int buf) {
    const int tx = tile % tiles_x, y0 = ((tile / tiles_x) % tiles_y) * R, b = tile / (tiles_x * tiles_y);
    const int x0 = tx * kM;
    mbar_expect_tx(&bar_load[buf], (R + 2) * KC * kPix * 16);
    for (int r = 0; r < R + 2; ++r) {
      const int yy = (y0 + r - 1 + H) % H;
      for (int c = 0; c < KC; ++c) {
        // columns x0 .. x0 + 129 of the padded row: pixels x0 - 1 .. x0 + 128
        const __nv_bfloat16* row = in + (((size_t)b * KC + c) * H + yy) * (size_t)(W + 2) * 8;
        bulk_g2s(sA(buf) + r * ROWB + c * kPix * 16, row + (size_t)x0 * 8, kPix * 16, &bar_load[buf]);
      }
    }
  };
  // the first tile's rows are on their way while the weights are copied
  if (threadIdx.x == 0) {
    mbar_init(&bar_load[0]);
    mbar_init(&bar_load[1]);
    mbar_init(&bar_mma);
    if ((int)blockIdx.x < tiles) issue_load(blockIdx.x, 0);
  }
  for (int i = threadIdx.x; i < WBYTES / 16; i += kThreadsTc)
    reinterpret_cast<uint4*>(sW)[i] = __ldg(reinterpret_cast<const uint4*>(wtc) + i);
  if (threadIdx.x < 32) s_bias[threadIdx.x] = (MODE != OUT_GRAD && threadIdx.x < cout_real) ? bias[threadIdx.x] : 0.f;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // weights: generic writes -> tensor-core reads
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t ph_load = 0u, ph_mma = 0u;      // parity of each load buffer (bit buf)
  uint32_t pending = (int)blockIdx.x < tiles ? 1u : 0u;   // load buffers with a copy in flight (bit buf)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int it = 0;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
    const int buf = it & 1;
    const int tx = tile % tiles_x, y0 = ((tile / tiles_x) % tiles_y) * R, b = tile / (tiles_x * tiles_y);
    const int x0 = tx * kM;
    bool ok = mbar_wait(&bar_load[buf], (ph_load >> buf) & 1u, err);
    ph_load ^= 1u << buf;
    pending &= ~(1u << buf);
    if (__syncthreads_or(!ok)) break;
    const int next = tile + gridDim.x;
    if (threadIdx.x == 0) {
      fence_after();
      constexpr uint32_t idesc = instr_desc(kM, COUT);
      // descriptors built once per tile; an operand further into shared
      // memory only adds its offset in 16-byte units to the start field
      // (shared addresses stay below 2^18 bytes, so the 14-bit field never carries)
      const uint64_t a0 = operand_desc(saddr(sA(buf)), kPix * 16, 128);
      const uint64_t b0 = operand_desc(saddr(sW), COUT * 16, 128);
#pragma unroll
      for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int dy = tap / 3, dx = tap % 3;
#pragma unroll
          for (int kk = 0; kk < KC / 2; ++kk) {
            const uint32_t a_off = (r + dy) * ROWB + (2 * kk) * kPix * 16 + dx * 16;
            const uint32_t b_off = (tap * KC + 2 * kk) * COUT * 16;
            mma(tmem + r * COUT, a0 + (a_off >> 4), b0 + (b_off >> 4), idesc, tap > 0 || kk > 0);
          }
        }
      }
      commit(&bar_mma);
      // the other buffer was last read by the previous tile's MMAs, which have completed
      if (next < tiles) issue_load(next, buf ^ 1);
    }
    if (next < tiles) pending |= 1u << (buf ^ 1);
    ok = mbar_wait(&bar_mma, ph_mma, err);
    ph_mma ^= 1u;
    fence_after();
    if (ok) {
      const int m = 32 * warp + lane;
      const uint32_t lanes = (uint32_t)(32 * warp) << 16;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int y = y0 + r;
        if constexpr (MODE == OUT_HIDDEN || MODE == OUT_GRAD) {
          float v[32];
          ld32(tmem + lanes + r * COUT, v);
#pragma unroll
          for (int j = 0; j < COUT / 8; ++j) {
            uint32_t packed[4];
            if constexpr (MODE == OUT_GRAD) {
              const uint4 mk = reinterpret_cast<const uint4*>(
                  mask + (((size_t)b * (COUT / 8) + j) * H + y) * (size_t)(W + 2) * 8)[x0 + m + 1];
              const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162*>(&mw[e]);
                const float lo = __low2float(m2) > 0.f ? v[8 * j + 2 * e] : 0.f;
                const float hi = __high2float(m2) > 0.f ? v[8 * j + 2 * e + 1] : 0.f;
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(lo, hi);
                packed[e] = *reinterpret_cast<const uint32_t*>(&h2);
              }
            } else {
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float lo = fmaxf(v[8 * j + 2 * e] + s_bias[8 * j + 2 * e], 0.f);
                const float hi = fmaxf(v[8 * j + 2 * e + 1] + s_bias[8 * j + 2 * e + 1], 0.f);
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(lo, hi);
                packed[e] = *reinterpret_cast<const uint32_t*>(&h2);
              }
            }
            const uint4 q = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            uint4* row = reinterpret_cast<uint4*>(out_bf + (((size_t)b * (COUT / 8) + j) * H + y) * (size_t)(W + 2) * 8);
            const int x = x0 + m;
            row[x + 1] = q;
            if (x == W - 1) row[0] = q;            // the halo copies of the row ends
            if (x == 0) row[W + 1] = q;
          }
        } else {
          float v[16];
          ld16(tmem + lanes + r * COUT, v);
          const float f0 = v[0] + s_bias[0], f1 = v[1] + s_bias[1];
          if constexpr (MODE == OUT_PLANES) {
            out_f[(((size_t)b * cout_real + 0) * H + y) * W + x0 + m] = f0;
            if (cout_real > 1) out_f[(((size_t)b * cout_real + 1) * H + y) * W + x0 + m] = f1;
          } else {
            const float s = sigma * amp[b];
            float2* e = field + ((size_t)b * H + y) * W + x0 + m;
            const float2 old = *e;
            *e = make_float2(fmaf(s, f0, old.x), fmaf(s, f1, old.y));
          }
        }
      }
    }
    fence_before();
    if (__syncthreads_or(!ok)) break;     // accumulators are free for the next tile
  }
  // leave no bulk copy in flight (only after a failed wait can one remain)
  if (threadIdx.x == 0)
    for (int k = 0; k < 2; ++k)
      if ((pending >> k) & 1u) mbar_wait(&bar_load[k], (ph_load >> k) & 1u, err);
  fence_before();
  __syncthreads();
  fence_after();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL) : "memory");
}

template <int CIN, int COUT>
constexpr size_t conv_tc_smem() {
  return ((size_t)(9 * (CIN / 8) * COUT * 16 + 127) & ~(size_t)127) + 2 * (size_t)(kRowsTc + 2) * (CIN / 8) * kPix * 16;
}

// store the two 16-byte chunks of one pixel into the padded chunk layout
// [b][2][y][W + 2][8], with the halo copies at the row ends
__device__ __forceinline__ void store_pixel_chunks(__nv_bfloat16* out, size_t b, int y, int x, int H, int W,
                                                   uint4 c0, uint4 c1) {
  uint4* r0 = reinterpret_cast<uint4*>(out + (((b * 2 + 0) * H + y) * (size_t)(W + 2)) * 8);
  uint4* r1 = reinterpret_cast<uint4*>(out + (((b * 2 + 1) * H + y) * (size_t)(W + 2)) * 8);
  r0[x + 1] = c0;
  r1[x + 1] = c1;
  if (x == W - 1) {
    r0[0] = c0;
    r1[0] = c1;
  }
  if (x == 0) {
    r0[W + 1] = c0;
    r1[W + 1] = c1;
  }
}

// packed FP32 input [b][cin][y][x] -> BF16 chunks (padded layout; channels >= cin zero)
__global__ void to_chunks(const float* __restrict__ x, int cin, int B, int H, int W, __nv_bfloat16* __restrict__ out) {
  const int hw = H * W;
  const size_t n = (size_t)B * hw;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / hw, p = i % hw;
    float c[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) c[k] = k < cin ? x[(b * cin + k) * hw + p] : 0.f;
    uint4 q[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint32_t packed[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(c[8 * j + 2 * e], c[8 * j + 2 * e + 1]);
        packed[e] = *reinterpret_cast<const uint32_t*>(&h2);
      }
      q[j] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
    store_pixel_chunks(out, b, (int)(p / W), (int)(p % W), H, W, q[0], q[1]);
  }
}

// apply: the field normalised by its RMS amplitude (and the index channel)
// straight into BF16 chunks [b][2][y][x][8]
__global__ void field_to_chunks(const float2* __restrict__ field, const __half* __restrict__ dn, float dn_scale,
                                const float* __restrict__ amp, int cin, int B, int H, int W,
                                __nv_bfloat16* __restrict__ out) {
  const int hw = H * W;
  const size_t n = (size_t)B * hw;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / hw, p = i % hw;
    const float inv = 1.0f / amp[b];
    const float2 e = field[i];
    const float c2 = (cin > 2 && dn) ? dn_scale * __half2float(dn[i]) : 0.f;
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(e.x * inv, e.y * inv);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(cin > 2 ? c2 : 0.f, 0.f);
    const uint32_t w0 = *reinterpret_cast<const uint32_t*>(&h0), w1 = *reinterpret_cast<const uint32_t*>(&h1);
    store_pixel_chunks(out, b, (int)(p / W), (int)(p % W), H, W, make_uint4(w0, w1, 0u, 0u), make_uint4(0u, 0u, 0u, 0u));
  }
}

// layer weights W[o][c][3][3] (FP32 values already rounded to BF16) -> [tap][c/8][o][8] BF16, zero padded
__global__ void pack_weights(const float* __restrict__ Wl, int cin, int cout, int cinp, int coutp,
                             __nv_bfloat16* __restrict__ out) {
  const int n = 9 * cinp * coutp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e = i % 8, o = (i / 8) % coutp, kc = (i / (8 * coutp)) % (cinp / 8), tap = i / (8 * coutp * (cinp / 8));
    const int c = kc * 8 + e;
    const float w = (o < cout && c < cin) ? Wl[((size_t)o * cin + c) * 9 + tap] : 0.f;
    out[i] = __float2bfloat16_rn(w);
  }
}

// Adjoint weights of layer W[o][c][3][3] for the data gradient: the
// convolution from the layer's output channels (o, padded to cinp) to its
// input channels (c, padded to coutp) with the taps mirrored,
// out[tap][o/8][c][o%8] = W[o][c][8 - tap], zero padded.
__global__ void pack_weights_adjoint(const float* __restrict__ Wl, int cin, int cout, int cinp, int coutp,
                                     __nv_bfloat16* __restrict__ out) {
  const int n = 9 * cinp * coutp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e = i % 8, c = (i / 8) % coutp, kc = (i / (8 * coutp)) % (cinp / 8), tap = i / (8 * coutp * (cinp / 8));
    const int o = kc * 8 + e;
    const float w = (o < cout && c < cin) ? Wl[((size_t)o * cin + c) * 9 + (8 - tap)] : 0.f;
    out[i] = __float2bfloat16_rn(w);
  }
}

// Weight and bias gradients of one 3x3 layer on the tensor cores,
//   dW[co][ci][tap] = sum_p dZ[co][p] X[ci][p + off(tap)],  db[co] = sum_p dZ[co][p],
// as D[m][n] = sum_k A[m][k] B[n][k] with m = tap CIN + ci (and m = 9 CIN a
// row of ones for the bias), n = co, and k running over the 128 pixels of
// one output row segment per step (all of the CTA's segments accumulate in
// tensor memory).  X and dZ are the BF16 chunk tensors of the forward and
// backward passes (CIN, COUT padded channel counts).  The threads transpose
// each segment into K-major operands in shared memory, core matrices of 8
// rows x 8 pixels (128 bytes) laid out [row / 8][pixel / 8][row % 8][pixel %
// 8], the x-shifted taps as their own rows; one thread issues the MMAs.  The
// CTA writes its sums to partial[blockIdx.x][P], P = cout_real cin_real 9 +
// cout_real, in the flat parameter order (W[co][ci][tap], then b[co]).
constexpr int kWgradThreads = 128;
template <int CIN, int COUT>
struct WgradShape {
  static constexpr int MROWS = 9 * CIN + 1;                     // taps x input channels, and the bias row
  static constexpr int MT = (MROWS + kM - 1) / kM;              // M tiles of 128 rows
  static constexpr int ABYTES = MT * kM * kM * 2;               // A: MT x 128 rows x 128 pixels, BF16
  static constexpr int BBYTES = COUT * kM * 2;                  // B: COUT rows x 128 pixels
  static constexpr int NCOL = tmem_cols(MT * COUT);
};
template <int CIN, int COUT>
constexpr size_t wgrad_tc_smem() {
  return (size_t)WgradShape<CIN, COUT>::ABYTES + WgradShape<CIN, COUT>::BBYTES + 128;
}

// element (row, pixel) of a K-major operand with 128 pixels per row
__device__ __forceinline__ int kmaj(int row, int k) { return ((row >> 3) * (kM / 8) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7); }

template <int CIN, int COUT>
__global__ void __launch_bounds__(kWgradThreads) wgrad_tc(const __nv_bfloat16* __restrict__ X,
                                                           const __nv_bfloat16* __restrict__ dZ, int cin_real,
                                                           int cout_real, float* __restrict__ partial, int B, int H,
                                                           int W, int* err) {
  using S = WgradShape<CIN, COUT>;
  static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 32, "padded channel counts");
  extern __shared__ __align__(128) unsigned char sm[];
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(sm);
  __nv_bfloat16* sB = reinterpret_cast<__nv_bfloat16*>(sm + S::ABYTES);
  __shared__ __align__(8) uint64_t bar_mma;
  __shared__ uint32_t tmem_base;
  const int tiles_x = W / kM, tiles = B * H * tiles_x;
  // rows that no segment overwrites: the bias row (ones) and the padding (zeros)
  const __nv_bfloat16 one = __float2bfloat16_rn(1.0f), zero = __float2bfloat16_rn(0.0f);
  for (int i = threadIdx.x; i < (S::MT * kM - 9 * CIN) * kM; i += kWgradThreads) {
    const int row = 9 * CIN + i / kM, k = i % kM;
    sA[kmaj(row, k)] = row == 9 * CIN ? one : zero;
  }
  if (threadIdx.x == 0) mbar_init(&bar_mma);
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(S::NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t ph = 0u;
  bool ok = true;
  int done = 0;
  for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++done) {
    const int tx = tile % tiles_x, y = (tile / tiles_x) % H, b = tile / (tiles_x * H);
    const int x0 = tx * kM;
    // A: rows tap CIN + ci, pixel k = X[ci][y + dy - 1][x0 + k + dx - 1] (padded column x0 + k + dx)
    for (int i = threadIdx.x; i < 3 * (CIN / 8) * (kM + 2); i += kWgradThreads) {
      const int col = i % (kM + 2), q = (i / (kM + 2)) % (CIN / 8), dy = i / ((kM + 2) * (CIN / 8));
      const int yy = (y + dy - 1 + H) % H;
      const uint4 v = reinterpret_cast<const uint4*>(X + (((size_t)b * (CIN / 8) + q) * H + yy) * (size_t)(W + 2) * 8)[x0 + col];
      const __nv_bfloat16* e8 = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int k = col - dx;
        if (k < 0 || k >= kM) continue;
        const int row0 = (dy * 3 + dx) * CIN + q * 8;
#pragma unroll
        for (int e = 0; e < 8; ++e) sA[kmaj(row0 + e, k)] = e8[e];
      }
    }
    // B: rows co, pixel k = dZ[co][y][x0 + k]
    for (int i = threadIdx.x; i < (COUT / 8) * kM; i += kWgradThreads) {
      const int k = i % kM, q = i / kM;
      const uint4 v = reinterpret_cast<const uint4*>(dZ + (((size_t)b * (COUT / 8) + q) * H + y) * (size_t)(W + 2) * 8)[x0 + k + 1];
      const __nv_bfloat16* e8 = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
      for (int e = 0; e < 8; ++e) sB[kmaj(q * 8 + e, k)] = e8[e];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_after();
      constexpr uint32_t idesc = instr_desc(kM, COUT);
      // K-major, no swizzle: the next 8 pixels (K) one core matrix further
      // (128 bytes), the next 8 rows (M or N) one row of core matrices further
      const uint64_t a0 = operand_desc(saddr(sA), 128, (kM / 8) * 128);
      const uint64_t b0 = operand_desc(saddr(sB), 128, (kM / 8) * 128);
#pragma unroll
      for (int t = 0; t < S::MT; ++t)
#pragma unroll
        for (int kb = 0; kb < kM / 16; ++kb) {
          const uint32_t a_off = t * kM * kM * 2 + kb * 2 * 128;
          const uint32_t b_off = kb * 2 * 128;
          mma(tmem + t * COUT, a0 + (a_off >> 4), b0 + (b_off >> 4), idesc, done > 0 || kb > 0);
        }
      commit(&bar_mma);
    }
    ok = mbar_wait(&bar_mma, ph, err);      // the operands are free again when the MMAs have completed
    ph ^= 1u;
    fence_after();
    if (__syncthreads_or(!ok)) break;
  }
  // read back: warp w holds rows 32w..32w+31 of each M tile
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = cout_real * cin_real * 9 + cout_real;
  float* out = partial + (size_t)blockIdx.x * P;
#pragma unroll
  for (int t = 0; t < S::MT; ++t) {
    float v[32];
    if (COUT == 32) ld32(tmem + ((uint32_t)(32 * warp) << 16) + t * COUT, v);
    else ld16(tmem + ((uint32_t)(32 * warp) << 16) + t * COUT, v);
    const int m = t * kM + 32 * warp + lane;
    for (int n = 0; n < cout_real; ++n) {
      const float g = (done > 0 && ok) ? v[n] : 0.f;
      if (m < 9 * CIN) {
        const int tap = m / CIN, ci = m % CIN;
        if (ci < cin_real) out[((size_t)n * cin_real + ci) * 9 + tap] = g;
      } else if (m == 9 * CIN) {
        out[(size_t)cout_real * cin_real * 9 + n] = g;
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::NCOL) : "memory");
}

}  // namespace tc

}  // namespace

struct bpm_corrector_s {
  int cin = 2, maxb = 0, maxh = 0, maxw = 0;
  int P = 0;                       // parameter count
  int off[8] = {};                 // offsets of W1,b1,...,W4,b4 in the flat vector
  float *master = nullptr, *work = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  float *x = nullptr;              // packed input [B][cin][H][W] (apply path)
  float *z[4] = {}, *a[3] = {};    // pre-activations and activations
  float *d0 = nullptr, *d1 = nullptr;   // backpropagated gradients (ping-pong)
  float *partial = nullptr, *lpart = nullptr, *loss = nullptr, *outbuf = nullptr, *amp = nullptr;
  float* rms_part = nullptr;       // per-field partial sums of |E|^2
  size_t partial_floats = 0;
  int step = 0;
  float sigma = 1.0f;              // residual scale: out = x[:, :2] + sigma f(x)
  // tensor-core inference path
  int use_tc = 1;                  // inference on tcgen05 when the width is a multiple of 128
  __nv_bfloat16* xtc = nullptr;    // input as BF16 chunks [B][2][H][W][8]
  __nv_bfloat16* atc[3] = {};      // hidden activations as BF16 chunks [B][4][H][W][8]
  __nv_bfloat16* wtc[4] = {};      // layer weights [tap][c_in/8][c_out][8]
  // tensor-core training path
  int train_tc = 0;                // loss and gradients on tcgen05 when the width is a multiple of 128
  __nv_bfloat16* gtc[2] = {};      // data gradients of the hidden layers, BF16 chunks [B][4][H][W][8]
  __nv_bfloat16* g4tc = nullptr;   // gradient of the output layer, BF16 chunks [B][2][H][W][8]
  __nv_bfloat16* wadj[4] = {};     // adjoint weights of layers 2..4 [tap][c_out/8][c_in][8]
  int* err = nullptr;              // device error word (bounded waits)
  unsigned wver = 1, tcver = 0;    // versions of the working weights and of their packed copy
};

namespace {

int layer_in(const bpm_corrector_s* c, int l) { return l == 0 ? c->cin : kCh; }
int layer_out(int l) { return l == 3 ? 2 : kCh; }
int layer_in_padded(int l) { return l == 0 ? 16 : kCh; }
int layer_out_padded(int l) { return l == 3 ? 16 : kCh; }

template <class K>
int set_smem(K kernel, size_t bytes) {
  CORR_CU(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return BPM_OK;
}

int setup_attrs() {
  static bool done = false;
  if (done) return BPM_OK;
  int rc = 0;
  rc |= set_smem(corr_conv<2, kCh, false, true, false, true>, conv_smem<2, kCh>());
  rc |= set_smem(corr_conv<3, kCh, false, true, false, true>, conv_smem<3, kCh>());
  rc |= set_smem(corr_conv<kCh, kCh, false, true, false, true>, conv_smem<kCh, kCh>());
  rc |= set_smem(corr_conv<kCh, 2, false, true, false, false>, conv_smem<kCh, 2>());
  rc |= set_smem(corr_conv<2, kCh, true, false, true, false>, conv_smem<2, kCh>());
  rc |= set_smem(corr_conv<kCh, kCh, true, false, true, false>, conv_smem<kCh, kCh>());
  rc |= set_smem(corr_wgrad<2, kCh>, wgrad_smem<2, kCh>());
  rc |= set_smem(corr_wgrad<3, kCh>, wgrad_smem<3, kCh>());
  rc |= set_smem(corr_wgrad<kCh, kCh>, wgrad_smem<kCh, kCh>());
  rc |= set_smem(corr_wgrad<kCh, 2>, wgrad_smem<kCh, 2>());
  rc |= set_smem(tc::conv_tc<16, kCh, tc::OUT_HIDDEN>, tc::conv_tc_smem<16, kCh>());
  rc |= set_smem(tc::conv_tc<kCh, kCh, tc::OUT_HIDDEN>, tc::conv_tc_smem<kCh, kCh>());
  rc |= set_smem(tc::conv_tc<kCh, 16, tc::OUT_PLANES>, tc::conv_tc_smem<kCh, 16>());
  rc |= set_smem(tc::conv_tc<kCh, 16, tc::OUT_FIELD>, tc::conv_tc_smem<kCh, 16>());
  rc |= set_smem(tc::conv_tc<16, kCh, tc::OUT_GRAD>, tc::conv_tc_smem<16, kCh>());
  rc |= set_smem(tc::conv_tc<kCh, kCh, tc::OUT_GRAD>, tc::conv_tc_smem<kCh, kCh>());
  rc |= set_smem(tc::wgrad_tc<kCh, 16>, tc::wgrad_tc_smem<kCh, 16>());
  rc |= set_smem(tc::wgrad_tc<kCh, kCh>, tc::wgrad_tc_smem<kCh, kCh>());
  rc |= set_smem(tc::wgrad_tc<16, kCh>, tc::wgrad_tc_smem<16, kCh>());
  if (rc) return BPM_ERR_CUDA;
  done = true;
  return BPM_OK;
}

int check_dims(const bpm_corrector_s* c, int batch, int h, int w) {
  if (batch < 1 || batch > c->maxb || h < 16 || w < 16 || h % 16 || w % 16 || (size_t)h * w > (size_t)c->maxh * c->maxw)
    return cfail(BPM_ERR_ARG, "batch must be in [1, %d]; h, w multiples of 16 with h*w <= %d*%d", c->maxb,
                 c->maxh, c->maxw);
  return BPM_OK;
}

// forward pass from the packed input x: fills z[0..3], a[0..2]
int forward(bpm_corrector_s* c, const float* x, int batch, int h, int w, cudaStream_t s) {
  dim3 grid(w / kTile, h / kTile, batch);
  const float* W1 = c->work + c->off[0];
  if (c->cin == 2)
    corr_conv<2, kCh, false, true, false, true><<<grid, 256, conv_smem<2, kCh>(), s>>>(
        x, W1, c->work + c->off[1], nullptr, c->z[0], c->a[0], h, w);
  else
    corr_conv<3, kCh, false, true, false, true><<<grid, 256, conv_smem<3, kCh>(), s>>>(
        x, W1, c->work + c->off[1], nullptr, c->z[0], c->a[0], h, w);
  for (int l = 1; l < 3; ++l)
    corr_conv<kCh, kCh, false, true, false, true><<<grid, 256, conv_smem<kCh, kCh>(), s>>>(
        c->a[l - 1], c->work + c->off[2 * l], c->work + c->off[2 * l + 1], nullptr, c->z[l], c->a[l], h, w);
  corr_conv<kCh, 2, false, true, false, false><<<grid, 256, conv_smem<kCh, 2>(), s>>>(
      c->a[2], c->work + c->off[6], c->work + c->off[7], nullptr, c->z[3], nullptr, h, w);
  CORR_CU(cudaGetLastError());
  return BPM_OK;
}

// BF16 copies of the working weights in the tensor-core layout (and the
// adjoint weights of layers 2..4 for the data gradients), refreshed when the
// working weights have changed
void ensure_tc_weights(bpm_corrector_s* c, cudaStream_t s) {
  if (c->tcver == c->wver) return;
  for (int l = 0; l < 4; ++l) {
    const int n = 9 * layer_in_padded(l) * layer_out_padded(l);
    tc::pack_weights<<<(n + 255) / 256, 256, 0, s>>>(c->work + c->off[2 * l], layer_in(c, l), layer_out(l),
                                                      layer_in_padded(l), layer_out_padded(l), c->wtc[l]);
    if (l > 0)
      tc::pack_weights_adjoint<<<(n + 255) / 256, 256, 0, s>>>(c->work + c->off[2 * l], layer_in(c, l), layer_out(l),
                                                                layer_out_padded(l), layer_in_padded(l), c->wadj[l]);
  }
  c->tcver = c->wver;
}

// the three hidden layers on the tensor cores: xtc -> atc[0] -> atc[1] -> atc[0]
int hidden_tc(bpm_corrector_s* c, int batch, int h, int w, int grid, cudaStream_t s) {
  tc::conv_tc<16, kCh, tc::OUT_HIDDEN><<<grid, tc::kThreadsTc, tc::conv_tc_smem<16, kCh>(), s>>>(
      c->xtc, c->wtc[0], c->work + c->off[1], kCh, c->atc[0], nullptr, nullptr, nullptr, 0.f, batch, h, w, c->err);
  tc::conv_tc<kCh, kCh, tc::OUT_HIDDEN><<<grid, tc::kThreadsTc, tc::conv_tc_smem<kCh, kCh>(), s>>>(
      c->atc[0], c->wtc[1], c->work + c->off[3], kCh, c->atc[1], nullptr, nullptr, nullptr, 0.f, batch, h, w, c->err);
  tc::conv_tc<kCh, kCh, tc::OUT_HIDDEN><<<grid, tc::kThreadsTc, tc::conv_tc_smem<kCh, kCh>(), s>>>(
      c->atc[1], c->wtc[2], c->work + c->off[5], kCh, c->atc[0], nullptr, nullptr, nullptr, 0.f, batch, h, w, c->err);
  CORR_CU(cudaGetLastError());
  return BPM_OK;
}

int tc_grid(int batch, int h, int w) {
  const int tiles = batch * (h / tc::kRowsTc) * (w / tc::kM);
  return std::max(1, std::min(tiles, 148 * 2));
}

// forward pass on the tensor cores (inference): z[3] = f(x) before the
// residual, from the packed FP32 input; activations BF16, accumulation FP32
int forward_tc(bpm_corrector_s* c, const float* x, int batch, int h, int w, cudaStream_t s) {
  ensure_tc_weights(c, s);
  const int hw = h * w;
  tc::to_chunks<<<grid_for((size_t)batch * hw), 256, 0, s>>>(x, c->cin, batch, h, w, c->xtc);
  const int grid = tc_grid(batch, h, w);
  int rc = hidden_tc(c, batch, h, w, grid, s);
  if (rc) return rc;
  tc::conv_tc<kCh, 16, tc::OUT_PLANES><<<grid, tc::kThreadsTc, tc::conv_tc_smem<kCh, 16>(), s>>>(
      c->atc[0], c->wtc[3], c->work + c->off[7], 2, nullptr, c->z[3], nullptr, nullptr, 0.f, batch, h, w, c->err);
  CORR_CU(cudaGetLastError());
  return BPM_OK;
}

// apply on the tensor cores: normalised field (and index) straight into BF16
// chunks, the network, and the residual update of the field in place
int apply_tc(bpm_corrector_s* c, float2* field, const __half* dn, float dn_scale, int h, int w, cudaStream_t s) {
  ensure_tc_weights(c, s);
  const int hw = h * w;
  tc::field_to_chunks<<<grid_for((size_t)hw), 256, 0, s>>>(field, dn, dn_scale, c->amp, c->cin, 1, h, w, c->xtc);
  const int grid = tc_grid(1, h, w);
  int rc = hidden_tc(c, 1, h, w, grid, s);
  if (rc) return rc;
  tc::conv_tc<kCh, 16, tc::OUT_FIELD><<<grid, tc::kThreadsTc, tc::conv_tc_smem<kCh, 16>(), s>>>(
      c->atc[0], c->wtc[3], c->work + c->off[7], 2, nullptr, nullptr, field, c->amp, c->sigma, 1, h, w, c->err);
  CORR_CU(cudaGetLastError());
  return BPM_OK;
}

// inference forward: the tensor-core path when enabled and the width allows it
int forward_infer(bpm_corrector_s* c, const float* x, int batch, int h, int w, cudaStream_t s) {
  if (c->use_tc && w % tc::kM == 0) return forward_tc(c, x, batch, h, w, s);
  return forward(c, x, batch, h, w, s);
}

// loss and full gradient (into c->grad) for packed x and target [B][2][H][W]
int loss_grad(bpm_corrector_s* c, const float* x, const float* target, int batch, int h, int w, cudaStream_t s) {
  int rc = forward(c, x, batch, h, w, s);
  if (rc) return rc;
  const int hw = h * w;
  const int lblocks = 256;
  corr_loss<<<lblocks, 256, 0, s>>>(x, c->cin, c->z[3], c->sigma, target, c->d0, c->lpart, batch, hw);
  corr_sum<<<1, 256, 0, s>>>(c->lpart, lblocks, 1.0f / (float)((size_t)batch * 2 * hw), c->loss);
  dim3 grid(w / kTile, h / kTile, batch);
  const int tiles = (w / kTile) * (h / kTile) * batch;
  // layer 4: weight gradient from A3 and dZ4 (d0); dZ3 = W4^T dZ4 masked by Z3 -> d1
  corr_wgrad<kCh, 2><<<grid, 256, wgrad_smem<kCh, 2>(), s>>>(c->a[2], c->d0, c->partial, h, w);
  corr_reduce<<<(2 * kCh * 9 + 2 + 255) / 256, 256, 0, s>>>(c->partial, tiles, 2 * kCh * 9 + 2, c->grad + c->off[6]);
  corr_conv<2, kCh, true, false, true, false><<<grid, 256, conv_smem<2, kCh>(), s>>>(
      c->d0, c->work + c->off[6], nullptr, c->z[2], c->d1, nullptr, h, w);
  float* dcur = c->d1;
  float* dnext = c->d0;
  for (int l = 2; l >= 1; --l) {
    // weight gradient of layer l+1 (0-based l) from A_{l} and dZ_{l+1}
    corr_wgrad<kCh, kCh><<<grid, 256, wgrad_smem<kCh, kCh>(), s>>>(c->a[l - 1], dcur, c->partial, h, w);
    corr_reduce<<<(kCh * kCh * 9 + kCh + 255) / 256, 256, 0, s>>>(c->partial, tiles, kCh * kCh * 9 + kCh,
                                                                   c->grad + c->off[2 * l]);
    corr_conv<kCh, kCh, true, false, true, false><<<grid, 256, conv_smem<kCh, kCh>(), s>>>(
        dcur, c->work + c->off[2 * l], nullptr, c->z[l - 1], dnext, nullptr, h, w);
    std::swap(dcur, dnext);
  }
  const int P1 = kCh * c->cin * 9 + kCh;
  if (c->cin == 2)
    corr_wgrad<2, kCh><<<grid, 256, wgrad_smem<2, kCh>(), s>>>(x, dcur, c->partial, h, w);
  else
    corr_wgrad<3, kCh><<<grid, 256, wgrad_smem<3, kCh>(), s>>>(x, dcur, c->partial, h, w);
  corr_reduce<<<(P1 + 255) / 256, 256, 0, s>>>(c->partial, tiles, P1, c->grad + c->off[0]);
  CORR_CU(cudaGetLastError());
  return BPM_OK;
}

// Loss and full gradient on the tensor cores: the forward pass keeps every
// layer's BF16 chunk activations (xtc, atc[0..2]), the output layer's FP32
// planes go through the loss kernel, then per layer from the top the weight
// and bias gradients (wgrad_tc, summed over CTAs in a fixed order) and the
// data gradient of the layer below (the adjoint convolution with the ReLU
// mask, OUT_GRAD), all with BF16 operands and FP32 accumulation.
int loss_grad_tc(bpm_corrector_s* c, const float* x, const float* target, int batch, int h, int w, cudaStream_t s) {
  ensure_tc_weights(c, s);
  const int hw = h * w;
  tc::to_chunks<<<grid_for((size_t)batch * hw), 256, 0, s>>>(x, c->cin, batch, h, w, c->xtc);
  const int grid = tc_grid(batch, h, w);
  tc::conv_tc<16, kCh, tc::OUT_HIDDEN><<<grid, tc::kThreadsTc, tc::conv_tc_smem<16, kCh>(), s>>>(
      c->xtc, c->wtc[0], c->work + c->off[1], kCh, c->atc[0], nullptr, nullptr, nullptr, 0.f, batch, h, w, c->err);
  for (int l = 1; l < 3; ++l)
    tc::conv_tc<kCh, kCh, tc::OUT_HIDDEN><<<grid, tc::kThreadsTc, tc::conv_tc_smem<kCh, kCh>(), s>>>(
        c->atc[l - 1], c->wtc[l], c->work + c->off[2 * l + 1], kCh, c->atc[l], nullptr, nullptr, nullptr, 0.f, batch, h,
        w, c->err);
  tc::conv_tc<kCh, 16, tc::OUT_PLANES><<<grid, tc::kThreadsTc, tc::conv_tc_smem<kCh, 16>(), s>>>(
      c->atc[2], c->wtc[3], c->work + c->off[7], 2, nullptr, c->z[3], nullptr, nullptr, 0.f, batch, h, w, c->err);
  const int lblocks = 256;
  corr_loss<<<lblocks, 256, 0, s>>>(x, c->cin, c->z[3], c->sigma, target, c->d0, c->lpart, batch, hw);
  corr_sum<<<1, 256, 0, s>>>(c->lpart, lblocks, 1.0f / (float)((size_t)batch * 2 * hw), c->loss);
  tc::to_chunks<<<grid_for((size_t)batch * hw), 256, 0, s>>>(c->d0, 2, batch, h, w, c->g4tc);
  const int wtiles = batch * h * (w / tc::kM);
  const int wgrid = std::max(1, std::min(wtiles, 148));
  auto reduce = [&](int P, float* dst) {
    corr_reduce<<<(P + 255) / 256, 256, 0, s>>>(c->partial, wgrid, P, dst);
  };
  // layer 4: gradients from A3 and dZ4; dZ3 = adjoint(dZ4) masked by A3
  tc::wgrad_tc<kCh, 16><<<wgrid, tc::kWgradThreads, tc::wgrad_tc_smem<kCh, 16>(), s>>>(
      c->atc[2], c->g4tc, kCh, 2, c->partial, batch, h, w, c->err);
  reduce(2 * kCh * 9 + 2, c->grad + c->off[6]);
  tc::conv_tc<16, kCh, tc::OUT_GRAD><<<grid, tc::kThreadsTc, tc::conv_tc_smem<16, kCh>(), s>>>(
      c->g4tc, c->wadj[3], nullptr, kCh, c->gtc[0], nullptr, nullptr, nullptr, 0.f, batch, h, w, c->err, c->atc[2]);
  // layers 3 and 2: gradients from A_{l-1} and dZ_l; dZ_{l-1} = adjoint(dZ_l) masked by A_{l-1}
  int cur = 0;
  for (int l = 2; l >= 1; --l) {
    tc::wgrad_tc<kCh, kCh><<<wgrid, tc::kWgradThreads, tc::wgrad_tc_smem<kCh, kCh>(), s>>>(
        c->atc[l - 1], c->gtc[cur], kCh, kCh, c->partial, batch, h, w, c->err);
    reduce(kCh * kCh * 9 + kCh, c->grad + c->off[2 * l]);
    tc::conv_tc<kCh, kCh, tc::OUT_GRAD><<<grid, tc::kThreadsTc, tc::conv_tc_smem<kCh, kCh>(), s>>>(
        c->gtc[cur], c->wadj[l], nullptr, kCh, c->gtc[cur ^ 1], nullptr, nullptr, nullptr, 0.f, batch, h, w, c->err,
        c->atc[l - 1]);
    cur ^= 1;
  }
  // layer 1: gradients from the input and dZ1
  tc::wgrad_tc<16, kCh><<<wgrid, tc::kWgradThreads, tc::wgrad_tc_smem<16, kCh>(), s>>>(
      c->xtc, c->gtc[cur], c->cin, kCh, c->partial, batch, h, w, c->err);
  reduce(kCh * c->cin * 9 + kCh, c->grad + c->off[0]);
  CORR_CU(cudaGetLastError());
  return BPM_OK;
}

// the training engine for this batch: tensor cores when enabled and the
// width allows it, else the FP32 pipes
int loss_grad_any(bpm_corrector_s* c, const float* x, const float* target, int batch, int h, int w, cudaStream_t s) {
  if (c->train_tc && w % tc::kM == 0 && h % tc::kRowsTc == 0) return loss_grad_tc(c, x, target, batch, h, w, s);
  return loss_grad(c, x, target, batch, h, w, s);
}

}  // namespace

extern "C" int bpm_corrector_create(bpm_corrector_t* out, int in_channels, int max_batch, int max_h, int max_w,
                                    cudaStream_t stream) {
  if (!out) return cfail(BPM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (in_channels != 2 && in_channels != 3) return cfail(BPM_ERR_ARG, "in_channels must be 2 or 3");
  if (max_batch < 1 || max_h < 16 || max_w < 16 || max_h % 16 || max_w % 16 || max_h > 4096 || max_w > 4096)
    return cfail(BPM_ERR_ARG, "max_batch >= 1; max_h, max_w multiples of 16 in [16, 4096]");
  int rc = setup_attrs();
  if (rc) return cfail(rc, "could not set kernel attributes");
  bpm_corrector_s* c = new (std::nothrow) bpm_corrector_s;
  if (!c) return cfail(BPM_ERR_ARG, "out of host memory");
  c->cin = in_channels;
  c->maxb = max_batch;
  c->maxh = max_h;
  c->maxw = max_w;
  int k = 0;
  for (int l = 0; l < 4; ++l) {
    c->off[2 * l] = k;
    k += layer_out(l) * layer_in(c, l) * 9;
    c->off[2 * l + 1] = k;
    k += layer_out(l);
  }
  c->P = k;
  const size_t act = (size_t)max_batch * kCh * max_h * max_w;
  const size_t tiles = (size_t)max_batch * (max_h / kTile) * (max_w / kTile);
  // per-tile partials of the FP32 path, per-CTA partials of the tensor-core path (at most 148 CTAs)
  c->partial_floats = std::max(tiles, (size_t)148) * (size_t)(kCh * kCh * 9 + kCh);
  bool ok = true;
  auto alloc = [&](float** p, size_t n) {
    if (ok && cudaMalloc(p, n * sizeof(float)) != cudaSuccess) ok = false;
  };
  alloc(&c->master, c->P);
  alloc(&c->work, c->P);
  alloc(&c->m, c->P);
  alloc(&c->v, c->P);
  alloc(&c->grad, c->P);
  alloc(&c->x, (size_t)max_batch * 3 * max_h * max_w);
  for (int l = 0; l < 4; ++l) alloc(&c->z[l], act);
  for (int l = 0; l < 3; ++l) alloc(&c->a[l], act);
  alloc(&c->d0, act);
  alloc(&c->d1, act);
  alloc(&c->partial, c->partial_floats);
  alloc(&c->lpart, 256);
  alloc(&c->loss, 1);
  alloc(&c->outbuf, (size_t)max_batch * 2 * max_h * max_w);
  alloc(&c->amp, (size_t)max_batch);
  alloc(&c->rms_part, (size_t)max_batch * kRmsChunks);
  auto alloc_bf = [&](__nv_bfloat16** p, size_t n) {
    if (ok && cudaMalloc(p, n * sizeof(__nv_bfloat16)) != cudaSuccess) ok = false;
  };
  // padded rows (W + 2 pixels) for the tensor-core layout: h (w + 2) = h w + 2h
  // with h w <= max_h max_w and w >= 16, so at most 9/8 of max_h max_w
  const size_t pad_hw = (size_t)max_h * max_w + 2 * ((size_t)max_h * max_w / 16);
  const size_t act_pad = (size_t)max_batch * kCh * pad_hw;
  alloc_bf(&c->xtc, (size_t)max_batch * 16 * pad_hw);
  for (int k = 0; k < 3; ++k) alloc_bf(&c->atc[k], act_pad);
  alloc_bf(&c->gtc[0], act_pad);
  alloc_bf(&c->gtc[1], act_pad);
  alloc_bf(&c->g4tc, (size_t)max_batch * 16 * pad_hw);
  for (int l = 1; l < 4; ++l) alloc_bf(&c->wadj[l], (size_t)9 * layer_in_padded(l) * layer_out_padded(l));
  for (int l = 0; l < 4; ++l) alloc_bf(&c->wtc[l], (size_t)9 * layer_in_padded(l) * layer_out_padded(l));
  if (ok && cudaMalloc(&c->err, sizeof(int)) != cudaSuccess) ok = false;
  if (ok) cudaMemsetAsync(c->err, 0, sizeof(int), stream);
  if (!ok) {
    cudaGetLastError();
    bpm_corrector_free(c);
    return cfail(BPM_ERR_CUDA, "cudaMalloc failed for the corrector buffers");
  }
  cudaMemsetAsync(c->master, 0, c->P * sizeof(float), stream);
  cudaMemsetAsync(c->work, 0, c->P * sizeof(float), stream);
  cudaMemsetAsync(c->m, 0, c->P * sizeof(float), stream);
  cudaMemsetAsync(c->v, 0, c->P * sizeof(float), stream);
  if (cudaStreamSynchronize(stream) != cudaSuccess) {
    bpm_corrector_free(c);
    return cfail(BPM_ERR_CUDA, "initialisation failed");
  }
  *out = c;
  return BPM_OK;
}

extern "C" int bpm_corrector_param_count(bpm_corrector_t c) { return c ? c->P : BPM_ERR_ARG; }

extern "C" int bpm_corrector_set_residual_scale(bpm_corrector_t c, float sigma) {
  if (!c || !(sigma > 0) || !std::isfinite(sigma)) return cfail(BPM_ERR_ARG, "sigma must be positive and finite");
  c->sigma = sigma;
  return BPM_OK;
}

extern "C" int bpm_corrector_set_params(bpm_corrector_t c, const float* h_params, int n, cudaStream_t stream) {
  if (!c || !h_params || n != c->P) return cfail(BPM_ERR_ARG, "need the corrector and %d parameters", c ? c->P : 0);
  CORR_CU(cudaMemcpyAsync(c->master, h_params, n * sizeof(float), cudaMemcpyHostToDevice, stream));
  CORR_CU(cudaMemsetAsync(c->m, 0, n * sizeof(float), stream));
  CORR_CU(cudaMemsetAsync(c->v, 0, n * sizeof(float), stream));
  corr_round_bf16<<<(n + 255) / 256, 256, 0, stream>>>(c->master, c->work, n);
  CORR_CU(cudaGetLastError());
  CORR_CU(cudaStreamSynchronize(stream));
  c->step = 0;
  ++c->wver;
  return BPM_OK;
}

extern "C" int bpm_corrector_get_params(bpm_corrector_t c, float* h_params, int n, int which, cudaStream_t stream) {
  if (!c || !h_params || n != c->P) return cfail(BPM_ERR_ARG, "need the corrector and %d parameters", c ? c->P : 0);
  const float* src = which == 1 ? c->work : (which == 2 ? c->grad : c->master);
  CORR_CU(cudaMemcpyAsync(h_params, src, n * sizeof(float), cudaMemcpyDeviceToHost, stream));
  CORR_CU(cudaStreamSynchronize(stream));
  return BPM_OK;
}

extern "C" int bpm_corrector_forward(bpm_corrector_t c, const float* d_x, float* d_out, int batch, int h, int w,
                                     cudaStream_t stream) {
  if (!c || !d_x || !d_out) return cfail(BPM_ERR_ARG, "NULL argument");
  int rc = check_dims(c, batch, h, w);
  if (rc) return rc;
  rc = forward_infer(c, d_x, batch, h, w, stream);
  if (rc) return rc;
  corr_residual<<<grid_for((size_t)batch * 2 * h * w), 256, 0, stream>>>(d_x, c->cin, c->z[3], c->sigma, d_out,
                                                                         batch, h * w);
  CORR_CU(cudaGetLastError());
  return BPM_OK;
}

extern "C" int bpm_corrector_loss_grad(bpm_corrector_t c, const float* d_x, const float* d_target, int batch, int h,
                                       int w, float* h_loss, cudaStream_t stream) {
  if (!c || !d_x || !d_target) return cfail(BPM_ERR_ARG, "NULL argument");
  int rc = check_dims(c, batch, h, w);
  if (rc) return rc;
  rc = loss_grad_any(c, d_x, d_target, batch, h, w, stream);
  if (rc) return rc;
  if (h_loss) {
    CORR_CU(cudaMemcpyAsync(h_loss, c->loss, sizeof(float), cudaMemcpyDeviceToHost, stream));
    CORR_CU(cudaStreamSynchronize(stream));
  }
  return BPM_OK;
}

extern "C" int bpm_corrector_adam(bpm_corrector_t c, float lr, cudaStream_t stream) {
  if (!c || !(lr > 0)) return cfail(BPM_ERR_ARG, "need the corrector and lr > 0");
  c->step += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, c->step)), c2 = (float)(1.0 - std::pow(b2, c->step));
  corr_adam<<<(c->P + 255) / 256, 256, 0, stream>>>(c->master, c->work, c->m, c->v, c->grad, c->P, lr, (float)b1,
                                                    (float)b2, c1, c2, 1e-8f);
  CORR_CU(cudaGetLastError());
  ++c->wver;
  return BPM_OK;
}

extern "C" int bpm_corrector_train_step(bpm_corrector_t c, const float* d_x, const float* d_target, int batch, int h,
                                        int w, float lr, float* h_loss, cudaStream_t stream) {
  int rc = bpm_corrector_loss_grad(c, d_x, d_target, batch, h, w, h_loss, stream);
  if (rc) return rc;
  return bpm_corrector_adam(c, lr, stream);
}

extern "C" int bpm_corrector_pack(bpm_corrector_t c, const void* d_fields, const void* d_targets, const void* d_dn,
                                  float dn_scale, float* d_x, float* d_t, int batch, int h, int w,
                                  cudaStream_t stream) {
  if (!c || !d_fields || !d_x || (d_targets && !d_t)) return cfail(BPM_ERR_ARG, "NULL argument");
  if (batch < 1 || batch > c->maxb || h < 1 || w < 1) return cfail(BPM_ERR_ARG, "bad sizes (batch <= %d)", c->maxb);
  corr_field_rms_partial<<<dim3(kRmsChunks, batch), 256, 0, stream>>>(static_cast<const float2*>(d_fields), h * w,
                                                                     c->rms_part);
  corr_field_rms_final<<<batch, 32, 0, stream>>>(c->rms_part, h * w, c->amp);
  corr_pack<<<grid_for((size_t)batch * h * w), 256, 0, stream>>>(
      static_cast<const float2*>(d_fields), static_cast<const float2*>(d_targets), static_cast<const __half*>(d_dn),
      dn_scale, c->amp, d_x, d_t, c->cin, batch, h * w);
  CORR_CU(cudaGetLastError());
  return BPM_OK;
}

extern "C" int bpm_corrector_apply(bpm_corrector_t c, void* d_field, const void* d_dn, float dn_scale, int h, int w,
                                   cudaStream_t stream) {
  if (!c || !d_field) return cfail(BPM_ERR_ARG, "NULL argument");
  int rc = check_dims(c, 1, h, w);
  if (rc) return rc;
  corr_field_rms_partial<<<dim3(kRmsChunks, 1), 256, 0, stream>>>(static_cast<const float2*>(d_field), h * w,
                                                                 c->rms_part);
  corr_field_rms_final<<<1, 32, 0, stream>>>(c->rms_part, h * w, c->amp);
  if (c->use_tc && w % tc::kM == 0)
    return apply_tc(c, static_cast<float2*>(d_field), static_cast<const __half*>(d_dn), dn_scale, h, w, stream);
  corr_pack<<<grid_for((size_t)h * w), 256, 0, stream>>>(static_cast<const float2*>(d_field), nullptr,
                                                          static_cast<const __half*>(d_dn), dn_scale, c->amp, c->x,
                                                          nullptr, c->cin, 1, h * w);
  rc = forward_infer(c, c->x, 1, h, w, stream);
  if (rc) return rc;
  corr_residual<<<grid_for((size_t)2 * h * w), 256, 0, stream>>>(c->x, c->cin, c->z[3], c->sigma, c->outbuf, 1,
                                                                  h * w);
  corr_unpack<<<grid_for((size_t)h * w), 256, 0, stream>>>(c->outbuf, c->amp, static_cast<float2*>(d_field), 1,
                                                            h * w);
  CORR_CU(cudaGetLastError());
  return BPM_OK;
}

extern "C" int bpm_coarsen_index(const void* d_dn, int nz, int ny, int nx, int factor, void* d_out,
                                 cudaStream_t stream) {
  if (!d_dn || !d_out || nz < 0 || ny < 1 || nx < 1 || factor < 1) return cfail(BPM_ERR_ARG, "bad arguments");
  const int nzc = nz / factor;
  if (nzc == 0) return BPM_OK;
  const size_t plane = (size_t)nx * ny;
  coarsen_index<<<grid_for((size_t)nzc * plane), 256, 0, stream>>>(static_cast<const __half*>(d_dn), nzc, plane,
                                                                    factor, static_cast<__half*>(d_out));
  CORR_CU(cudaGetLastError());
  return BPM_OK;
}

extern "C" int bpm_corrector_set_tensor_cores(bpm_corrector_t c, int on) {
  if (!c) return cfail(BPM_ERR_ARG, "corrector is NULL");
  c->use_tc = on ? 1 : 0;
  return BPM_OK;
}

extern "C" int bpm_corrector_set_train_tensor_cores(bpm_corrector_t c, int on) {
  if (!c) return cfail(BPM_ERR_ARG, "corrector is NULL");
  c->train_tc = on ? 1 : 0;
  return BPM_OK;
}

extern "C" int bpm_corrector_check(bpm_corrector_t c, cudaStream_t stream) {
  if (!c) return cfail(BPM_ERR_ARG, "corrector is NULL");
  CORR_CU(cudaStreamSynchronize(stream));
  int e = 0;
  CORR_CU(cudaMemcpy(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) return cfail(e, "a tensor-core convolution gave up waiting for its data or its MMAs");
  return BPM_OK;
}

extern "C" int bpm_corrector_free(bpm_corrector_t c) {
  if (!c) return BPM_OK;
  float* bufs[] = {c->master, c->work, c->m, c->v, c->grad, c->x, c->z[0], c->z[1], c->z[2], c->z[3],
                   c->a[0], c->a[1], c->a[2], c->d0, c->d1, c->partial, c->lpart, c->loss, c->outbuf, c->amp};
  for (float* b : bufs) cudaFree(b);
  cudaFree(c->xtc);
  for (int k = 0; k < 3; ++k) cudaFree(c->atc[k]);
  cudaFree(c->gtc[0]);
  cudaFree(c->gtc[1]);
  cudaFree(c->g4tc);
  for (int l = 0; l < 4; ++l) {
    cudaFree(c->wtc[l]);
    cudaFree(c->wadj[l]);
  }
  cudaFree(c->err);
  cudaFree(c->rms_part);
  delete c;
  return BPM_OK;
}

extern "C" const char* bpm_corrector_last_error(void) { return g_corr_err.c_str(); }
