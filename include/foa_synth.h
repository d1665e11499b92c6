/*
 * foa_synth.h -- device generator of the synthetic snapshot sequences used by the benchmark and
 * the full-size tests.  It holds no part of the DMD method: it evaluates the modal synthesis
 *
 *   x_t[r] = sum_m F(r,m) T_f(r)[m] + noise_scale * xi(t, r)
 *
 * element by element with round-to-nearest operations in a fixed order, so that a host
 * evaluation of the same formula in the same precision gives identical values.  The paper has
 * no counterpart; its flow datasets are not available and are replaced by these sequences.
 *
 * F kinds: plane waves exp(i k.r) on a periodic grid of `axes` axes with G points each and
 * n_fields stacked fields (row r = ((f*G + i)*G + j)*G + k), built from per-axis (cos, sin)
 * tables; or Gaussian vectors from the Philox4x32-10 counter-based generator (Salmon et al.,
 * SC'11) with an Irwin-Hall(4) unit-variance transform.  Noise uses the same transform.
 *
 * dtype: FOA_DMD_F64 (FP64 arithmetic), FOA_DMD_F32 (FP32 arithmetic) or FOA_DMD_BF16 (FP32
 * arithmetic, result rounded to BF16).  All pointers are device pointers; tables and coef are
 * FP64 for FOA_DMD_F64 and FP32 otherwise.  Returns a foa_dmd_status.
 */
#ifndef FOA_SYNTH_H
#define FOA_SYNTH_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* tables: [axes][M][G][2] (cos, sin); coef: [n_fields][2M] time coefficients of snapshot t */
int foa_synth_waves(void *x_dev, int32_t dtype, int64_t n, int32_t axes, int32_t G, int32_t n_fields, int32_t M,
                    const void *tables, const void *coef, double noise_scale, uint32_t seed_noise, int64_t t,
                    void *cuda_stream);

/* coef: [M] time coefficients of snapshot t; mode entries are scaled by mode_scale */
int foa_synth_gauss(void *x_dev, int32_t dtype, int64_t n, int32_t M, uint32_t seed_modes, double mode_scale,
                    const void *coef, double noise_scale, uint32_t seed_noise, int64_t t, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
