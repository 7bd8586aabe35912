// bpm_aux_kernels.cuh - the library's non-templated kernels: plan tables
// (propagator, adapted-propagator rates), per-slice index means, multiplexed
// input scatter and pupil count, phase conjugation and PSF de-multiplexing.
// Included by bpm.cu only (the kernels are defined once).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bpm_args.cuh"

namespace bpmk {

// Mean index step of every slice (reading B): CTA z sums slice z0 + z of the
// FP16 volume (FP32 partial sums of at most M / kThreads values per thread,
// FP64 across the block) into delta[z].
__global__ void __launch_bounds__(kThreads) bpm_slice_mean_kernel(const __half* __restrict__ dn, size_t M,
                                                                  float* __restrict__ delta) {
  const __half* slice = dn + (size_t)blockIdx.x * M;
  float acc = 0.f;
  const size_t M8 = M / 8;   // 16-byte loads of 8 values (M is a multiple of 8)
  for (size_t i = threadIdx.x; i < M8; i += kThreads) {
    const uint4 u = __ldcs(reinterpret_cast<const uint4*>(slice) + i);
    const __half2* h = reinterpret_cast<const __half2*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __half22float2(h[k]);
      acc += f.x + f.y;
    }
  }
  for (size_t i = M8 * 8 + threadIdx.x; i < M; i += kThreads) acc += __half2float(slice[i]);
  __shared__ double part[kWarps];
  double d = acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += part[w];
    delta[blockIdx.x] = (float)(t / (double)M);
  }
}

// G = k0^2 n0 dz / kz0 per component (0 where the propagator is cut), laid out
// like ht ([kx][ky]); the cut is decided exactly as in bpm_build_ht_kernel.
__global__ void bpm_build_gt_kernel(float* gt, int nx, int ny, double dx, double dy, double dz, double lambda,
                                    double n0) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nx * ny) return;
  const int kyi = (int)(i % ny), kxi = (int)(i / ny);
  const int fx = kxi < (nx + 1) / 2 ? kxi : kxi - nx;
  const int fy = kyi < (ny + 1) / 2 ? kyi : kyi - ny;
  const double twopi = 6.283185307179586;
  const double k0 = __ddiv_rn(twopi, lambda);
  const double K = __dmul_rn(k0, n0);
  const double kx = __ddiv_rn(__dmul_rn(twopi, (double)fx), __dmul_rn((double)nx, dx));
  const double ky = __ddiv_rn(__dmul_rn(twopi, (double)fy), __dmul_rn((double)ny, dy));
  const double kz2 = __dsub_rn(__dsub_rn(__dmul_rn(K, K), __dmul_rn(kx, kx)), __dmul_rn(ky, ky));
  gt[i] = kz2 > 0.0 ? (float)(k0 * k0 * n0 * dz / sqrt(kz2)) : 0.f;
}

// Propagator table, transposed: ht[kx * ny + ky] = exp(i (kz - k0 n0) dz) / (nx ny)
// for kz^2 = (k0 n0)^2 - kx^2 - ky^2 > 0, else 0.  FP64 throughout; the
// cancellation-free form kz - k0 n0 = -k_perp^2 / (k0 n0 + kz) is used.
__global__ void bpm_build_ht_kernel(float2* ht, int nx, int ny, double dx, double dy, double dz, double lambda,
                                    double n0) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nx * ny) return;
  const int kyi = (int)(i % ny), kxi = (int)(i / ny);
  const int fx = kxi < (nx + 1) / 2 ? kxi : kxi - nx;
  const int fy = kyi < (ny + 1) / 2 ? kyi : kyi - ny;
  const double twopi = 6.283185307179586;
  const double K = __dmul_rn(__ddiv_rn(twopi, lambda), n0);
  const double kx = __ddiv_rn(__dmul_rn(twopi, (double)fx), __dmul_rn((double)nx, dx));
  const double ky = __ddiv_rn(__dmul_rn(twopi, (double)fy), __dmul_rn((double)ny, dy));
  const double kz2 = __dsub_rn(__dsub_rn(__dmul_rn(K, K), __dmul_rn(kx, kx)), __dmul_rn(ky, ky));
  float2 h = make_float2(0.f, 0.f);
  if (kz2 > 0.0) {
    const double kp2 = kx * kx + ky * ky;
    const double ph = -kp2 / (K + sqrt(kz2)) * dz;
    double sn, cs;
    sincos(ph, &sn, &cs);
    const double sc = 1.0 / ((double)nx * (double)ny);
    h = make_float2((float)(cs * sc), (float)(sn * sc));
  }
  ht[i] = h;
}

// Scatter emitters: out[iy][ix] += amp exp(i phase).  One thread per emitter.
__global__ void bpm_scatter_kernel(float2* field, int nx, int ny, const int* idx, const double* phase, int count,
                                   const unsigned long long* n_pupil) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  const double np = (double)*n_pupil;
  if (np <= 0.0) return;
  const double amp = sqrt((double)nx * (double)ny / np);
  double sn, cs;
  sincos(phase[j], &sn, &cs);
  float* p = reinterpret_cast<float*>(field + idx[j]);
  atomicAdd(p, (float)(amp * cs));
  atomicAdd(p + 1, (float)(amp * sn));
}

// Count DFT bins inside the pupil kin2 <= |k_perp|^2 <= kna2 that also propagate.
__global__ void bpm_pupil_count_kernel(int nx, int ny, double dx, double dy, double k0n0, double kin2, double kna2,
                                       unsigned long long* count) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  unsigned long long c = 0;
  if (i < (size_t)nx * ny) {
    const int x = (int)(i % nx), y = (int)(i / nx);
    const int fx = x < (nx + 1) / 2 ? x : x - nx, fy = y < (ny + 1) / 2 ? y : y - ny;
    const double kx = __ddiv_rn(__dmul_rn(6.283185307179586, (double)fx), __dmul_rn((double)nx, dx));
    const double ky = __ddiv_rn(__dmul_rn(6.283185307179586, (double)fy), __dmul_rn((double)ny, dy));
    const double kp2 = __dadd_rn(__dmul_rn(kx, kx), __dmul_rn(ky, ky));
    const double kz2 = __dsub_rn(__dmul_rn(k0n0, k0n0), kp2);
    c = (kp2 >= kin2 && kp2 <= kna2 && kz2 > 0.0) ? 1ull : 0ull;
  }
  // warp reduce, one atomic per warp
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// Phase conjugation of a field (time reversal of a monochromatic wave): E <- conj(E).
__global__ void bpm_conj_kernel(float2* E, size_t M) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
    float2 e = E[i];
    e.y = -e.y;
    E[i] = e;
  }
}

// Per-focus patches of an intensity window (PSF de-multiplexing): thread i
// of the grid-stride loop writes out[i], i = ((j pz + k) py + y) px + x, from
// voxel (iz_j - pz/2 + k, iy_j - py/2 + y, ix_j - px/2 + x) of the volume,
// laterally periodic (the grid's boundary condition); slices outside the
// window [w0, w0 + wnz) give 0.  foci: (ix, iy, iz) triples.
__global__ void bpm_demux_kernel(const float* __restrict__ I, int nx, int ny, int w0, int wnz, const int* __restrict__ foci,
                                 int n_foci, int px, int py, int pz, float* __restrict__ out) {
  const long long per = (long long)px * py * pz;
  const long long total = per * n_foci;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / per);
    long long r = i - (long long)j * per;
    const int k = (int)(r / ((long long)px * py));
    r -= (long long)k * px * py;
    const int y = (int)(r / px), x = (int)(r - (long long)y * px);
    const int z = foci[3 * j + 2] - pz / 2 + k - w0;
    float v = 0.f;
    if (z >= 0 && z < wnz) {
      const int yy = ((foci[3 * j + 1] - py / 2 + y) % ny + ny) % ny;
      const int xx = ((foci[3 * j] - px / 2 + x) % nx + nx) % nx;
      v = __ldcs(I + ((size_t)z * ny + yy) * nx + xx);
    }
    __stcs(out + i, v);
  }
}

}  // namespace bpmk
