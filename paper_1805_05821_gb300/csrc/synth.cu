// Device evaluation of the synthetic snapshot sequences (see include/foa_synth.h).  Every
// arithmetic operation is an explicit round-to-nearest intrinsic so the compiler cannot
// contract or reorder it; the host generator applies the same operations in the same order.
#include "api_internal.cuh"
#include "foa_synth.h"

namespace foa {

template <typename T> struct RN;
template <> struct RN<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float from_u24(uint32_t v) { return __uint2float_rn(v); }
};
template <> struct RN<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double from_u24(uint32_t v) { return __uint2double_rn(v); }
};

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// (u0+u1+u2+u3-2)*sqrt3 with u = (w >> 8) * 2^-24
template <typename T>
__device__ __forceinline__ T irwin_hall4(const uint32_t w[4], T sqrt3) {
  const T inv = T(1.0 / 16777216.0);
  T u[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) u[i] = RN<T>::mul(RN<T>::from_u24(w[i] >> 8), inv);
  T s = RN<T>::add(RN<T>::add(RN<T>::add(u[0], u[1]), u[2]), u[3]);
  return RN<T>::mul(RN<T>::sub(s, T(2)), sqrt3);
}

template <typename T, typename O>
__device__ __forceinline__ void store_out(O *x, int64_t r, T v);
template <>
__device__ __forceinline__ void store_out<double, double>(double *x, int64_t r, double v) { x[r] = v; }
template <>
__device__ __forceinline__ void store_out<float, float>(float *x, int64_t r, float v) { x[r] = v; }
template <>
__device__ __forceinline__ void store_out<float, __nv_bfloat16>(__nv_bfloat16 *x, int64_t r, float v) {
  x[r] = __float2bfloat16_rn(v);
}

template <typename T, typename O>
__global__ void synth_waves_kernel(O *x, int64_t n, int axes, int G, int nf, int M, const T *tables, const T *coef,
                                   T noise_scale, T sqrt3, uint32_t seed_noise, int64_t t) {
  extern __shared__ __align__(16) unsigned char smem[];
  T *cf = reinterpret_cast<T *>(smem);
  for (int i = threadIdx.x; i < nf * 2 * M; i += blockDim.x) cf[i] = coef[i];
  __syncthreads();
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += stride) {
    int idx[3];
    int64_t rem = r;
    for (int a = axes - 1; a >= 0; --a) {
      idx[a] = int(rem % G);
      rem /= G;
    }
    const int f = int(rem);
    const T *cff = cf + f * 2 * M;
    T acc = T(0);
    for (int m = 0; m < M; ++m) {
      const T *t0 = tables + (int64_t(0 * M + m) * G + idx[0]) * 2;
      T sr = t0[0], si = t0[1];
      for (int a = 1; a < axes; ++a) {
        const T *ta = tables + (int64_t(a * M + m) * G + idx[a]) * 2;
        const T br = ta[0], bi = ta[1];
        const T nr = RN<T>::sub(RN<T>::mul(sr, br), RN<T>::mul(si, bi));
        const T ni = RN<T>::add(RN<T>::mul(sr, bi), RN<T>::mul(si, br));
        sr = nr;
        si = ni;
      }
      acc = RN<T>::add(acc, RN<T>::mul(sr, cff[2 * m]));
      acc = RN<T>::add(acc, RN<T>::mul(si, cff[2 * m + 1]));
    }
    if (noise_scale != T(0)) {
      uint32_t c[4] = {uint32_t(r & 0xFFFFFFFFll), uint32_t(uint64_t(r) >> 32), uint32_t(t), 1u};
      philox4x32_10(c, seed_noise, 0x401Eu);
      acc = RN<T>::add(acc, RN<T>::mul(noise_scale, irwin_hall4<T>(c, sqrt3)));
    }
    store_out<T, O>(x, r, acc);
  }
}

template <typename T, typename O>
__global__ void synth_gauss_kernel(O *x, int64_t n, int M, uint32_t seed_modes, T mode_scale, const T *coef,
                                   T noise_scale, T sqrt3, uint32_t seed_noise, int64_t t) {
  extern __shared__ __align__(16) unsigned char smem[];
  T *cf = reinterpret_cast<T *>(smem);
  for (int i = threadIdx.x; i < M; i += blockDim.x) cf[i] = coef[i];
  __syncthreads();
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += stride) {
    T acc = T(0);
    for (int m = 0; m < M; ++m) {
      uint32_t c[4] = {uint32_t(r & 0xFFFFFFFFll), uint32_t(uint64_t(r) >> 32), uint32_t(m), 0u};
      philox4x32_10(c, seed_modes, 0x5EEDu);
      const T g = RN<T>::mul(irwin_hall4<T>(c, sqrt3), mode_scale);
      acc = RN<T>::add(acc, RN<T>::mul(g, cf[m]));
    }
    if (noise_scale != T(0)) {
      uint32_t c[4] = {uint32_t(r & 0xFFFFFFFFll), uint32_t(uint64_t(r) >> 32), uint32_t(t), 1u};
      philox4x32_10(c, seed_noise, 0x401Eu);
      acc = RN<T>::add(acc, RN<T>::mul(noise_scale, irwin_hall4<T>(c, sqrt3)));
    }
    store_out<T, O>(x, r, acc);
  }
}

static int synth_grid(int64_t n) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t g = (n + 255) / 256;
  if (g > int64_t(sms) * 16) g = int64_t(sms) * 16;
  return int(g < 1 ? 1 : g);
}

}  // namespace foa

using namespace foa;

extern "C" int foa_synth_waves(void *x_dev, int32_t dtype, int64_t n, int32_t axes, int32_t G, int32_t n_fields,
                               int32_t M, const void *tables, const void *coef, double noise_scale,
                               uint32_t seed_noise, int64_t t, void *cuda_stream) {
  if (!x_dev || !tables || !coef || n < 1 || axes < 1 || axes > 3 || G < 1 || n_fields < 1 || M < 1)
    return FOA_DMD_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int grid = synth_grid(n);
  const double sq3 = 1.7320508075688772;
  if (dtype == FOA_DMD_F64) {
    const size_t smem = size_t(n_fields) * 2 * M * 8;
    synth_waves_kernel<double, double><<<grid, 256, smem, s>>>(static_cast<double *>(x_dev), n, axes, G, n_fields, M,
                                                              static_cast<const double *>(tables),
                                                              static_cast<const double *>(coef), noise_scale, sq3,
                                                              seed_noise, t);
  } else {
    const size_t smem = size_t(n_fields) * 2 * M * 4;
    if (dtype == FOA_DMD_F32)
      synth_waves_kernel<float, float><<<grid, 256, smem, s>>>(
          static_cast<float *>(x_dev), n, axes, G, n_fields, M, static_cast<const float *>(tables),
          static_cast<const float *>(coef), float(noise_scale), float(sq3), seed_noise, t);
    else
      synth_waves_kernel<float, __nv_bfloat16><<<grid, 256, smem, s>>>(
          static_cast<__nv_bfloat16 *>(x_dev), n, axes, G, n_fields, M, static_cast<const float *>(tables),
          static_cast<const float *>(coef), float(noise_scale), float(sq3), seed_noise, t);
  }
  return cuda_status(cudaGetLastError());
}

extern "C" int foa_synth_gauss(void *x_dev, int32_t dtype, int64_t n, int32_t M, uint32_t seed_modes,
                               double mode_scale, const void *coef, double noise_scale, uint32_t seed_noise,
                               int64_t t, void *cuda_stream) {
  if (!x_dev || !coef || n < 1 || M < 1) return FOA_DMD_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int grid = synth_grid(n);
  const double sq3 = 1.7320508075688772;
  if (dtype == FOA_DMD_F64) {
    synth_gauss_kernel<double, double><<<grid, 256, size_t(M) * 8, s>>>(
        static_cast<double *>(x_dev), n, M, seed_modes, mode_scale, static_cast<const double *>(coef), noise_scale,
        sq3, seed_noise, t);
  } else if (dtype == FOA_DMD_F32) {
    synth_gauss_kernel<float, float><<<grid, 256, size_t(M) * 4, s>>>(
        static_cast<float *>(x_dev), n, M, seed_modes, float(mode_scale), static_cast<const float *>(coef),
        float(noise_scale), float(sq3), seed_noise, t);
  } else {
    synth_gauss_kernel<float, __nv_bfloat16><<<grid, 256, size_t(M) * 4, s>>>(
        static_cast<__nv_bfloat16 *>(x_dev), n, M, seed_modes, float(mode_scale), static_cast<const float *>(coef),
        float(noise_scale), float(sq3), seed_noise, t);
  }
  return cuda_status(cudaGetLastError());
}
