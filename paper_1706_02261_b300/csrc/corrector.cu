// corrector.cu - learned coarse-step corrector: training and inference kernels.
//
// A 4-layer 3x3 convolutional network (C_in -> 32 -> 32 -> 32 -> 2, ReLU
// between, circular padding, residual output out = x[:, :2] + f(x)) corrects
// the field after each coarse split-step of length 4 dz.  Weights are kept as
// FP32 masters with Adam moments; the convolutions use the BF16-rounded
// weights (stored as float) and accumulate in FP32.  Layout of every activation
// tensor: [batch][channel][y][x] float; H and W multiples of 16.
//
// Kernels (all direct convolutions on the FP32 pipes):
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
__global__ void corr_field_rms(const float2* __restrict__ field, int hw, float* __restrict__ amp) {
  __shared__ double red[256];
  const float2* f = field + (size_t)blockIdx.x * hw;
  double s = 0.0;
  for (int p = threadIdx.x; p < hw; p += 256) s += (double)f[p].x * f[p].x + (double)f[p].y * f[p].y;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double a = sqrt(red[0] / hw);
    amp[blockIdx.x] = a > 0.0 ? (float)a : 1.0f;
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
  size_t partial_floats = 0;
  int step = 0;
  float sigma = 1.0f;              // residual scale: out = x[:, :2] + sigma f(x)
};

namespace {

int layer_in(const bpm_corrector_s* c, int l) { return l == 0 ? c->cin : kCh; }
int layer_out(int l) { return l == 3 ? 2 : kCh; }

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
  c->partial_floats = tiles * (size_t)(kCh * kCh * 9 + kCh);
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
  rc = forward(c, d_x, batch, h, w, stream);
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
  rc = loss_grad(c, d_x, d_target, batch, h, w, stream);
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
  corr_field_rms<<<batch, 256, 0, stream>>>(static_cast<const float2*>(d_fields), h * w, c->amp);
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
  corr_field_rms<<<1, 256, 0, stream>>>(static_cast<const float2*>(d_field), h * w, c->amp);
  corr_pack<<<grid_for((size_t)h * w), 256, 0, stream>>>(static_cast<const float2*>(d_field), nullptr,
                                                          static_cast<const __half*>(d_dn), dn_scale, c->amp, c->x,
                                                          nullptr, c->cin, 1, h * w);
  rc = forward(c, c->x, 1, h, w, stream);
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

extern "C" int bpm_corrector_free(bpm_corrector_t c) {
  if (!c) return BPM_OK;
  float* bufs[] = {c->master, c->work, c->m, c->v, c->grad, c->x, c->z[0], c->z[1], c->z[2], c->z[3],
                   c->a[0], c->a[1], c->a[2], c->d0, c->d1, c->partial, c->lpart, c->loss, c->outbuf, c->amp};
  for (float* b : bufs) cudaFree(b);
  delete c;
  return BPM_OK;
}

extern "C" const char* bpm_corrector_last_error(void) { return g_corr_err.c_str(); }
