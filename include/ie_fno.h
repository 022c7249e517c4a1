/*
 * ie_fno.h — C ABI of the Fourier-neural-operator (FNO) warm start for the sub-domain GMRES solves.
 *
 * This network is an extension of the method, not part of the paper. The paper warm-starts each
 * block solve from the previous sweep's field (Algorithm 1, the adaptive block tolerance of
 * Section 2.3); in the first sweep the block solution starts from its right-hand side. The FNO
 * replaces that first guess by a prediction of the block solution of (I - G dsigma) E = b (eq. 8
 * restricted to an n^3 sub-domain) from the conductivity contrast and b. Restarted GMRES from the
 * predicted field remains the solver; ie_solve keeps E = b when the prediction's residual is not
 * smaller (see ie_set_initial_field_dev in ie.h).
 *
 * Network (channels-last activations, (batch, z, y, x, channel), cell index (z n + y) n + x):
 *     lift     v_0 = a P + p                                   (cin -> width)
 *     layers   v_{l+1} = act(v_l W_l + w_l + K_l v_l)            act = GELU (erf form), none after the last
 *     spectral K_l v = S(R_l * T v): T the DFT of the real field truncated to kz in [0, m) and
 *              ky, kx in [0, m) U [n-m, n); R_l one complex width x width matrix per retained mode;
 *              S the matching real inverse (weight 2 for kz > 0, factor n^-3)
 *     head     u = GELU(v_L Q1 + q1) Q2 + q2                     (width -> hidden -> cout)
 * Parameters travel as one FP32 vector in this order and layout:
 *     P [cin][width], p [width], W_0..W_{L-1} [width][width], w_0..w_{L-1} [width],
 *     R_0..R_{L-1} complex interleaved [m][2m][2m][width (in)][width (out)], Q1 [width][hidden],
 *     q1 [hidden], Q2 [hidden][cout], q2 [cout].
 * Storage: parameters, gradients and Adam moments in FP32; saved activations and the spectral weights
 * used by the kernels in BF16 (storage 1) or FP32 (storage 0); every sum accumulates in FP32.
 *
 * Warm-start encoding (cin = 12, cout = 6) for a sub-domain of N = n^3 cells:
 *     a[p] = (dsigma_xx, yy, zz, xy, xz, yz at p (S/m); Re, Im of b_x, b_y, b_z at p times sqrt(N)/|b|)
 *     target / prediction u[p] = Re, Im of (E - b)_{x,y,z} at p times sqrt(N)/|b|
 * so that E ~ b + |b|/sqrt(N) u.
 *
 * Conventions: device pointers are CUDA device memory of the current device, owned by the caller;
 * work runs on the network's stream (ie_fno_set_stream; default the legacy default stream) and
 * calls that take device pointers do not synchronise. Fields are complex128 [3][n][n][n]
 * interleaved; sigma6 is [n][n][n][6] absolute conductivity (ie.h conventions). Every call returns an
 * ie_status: IE_EINVAL for bad arguments, IE_ENOMEM for failed allocation, IE_ECUDA for a CUDA error
 * (the message is in ie_fno_last_error; the network should then be destroyed).
 */
#ifndef IE_GB300_FNO_H
#define IE_GB300_FNO_H

#include "ie.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ie_fno ie_fno;

/* Create a network for n^3 inputs (2 <= n <= 256), modes m (1 <= 2m <= n), width, layers, cin, cout,
 * hidden (each <= 128, every weight matrix at most 4096 entries), batch_max samples per call and
 * activation storage (0 FP32, 1 BF16). Parameters start at zero; load them with ie_fno_set_params. */
ie_status ie_fno_create(int32_t n, int32_t modes, int32_t width, int32_t layers, int32_t cin, int32_t cout,
                        int32_t hidden, int32_t batch_max, int32_t storage, ie_fno** out);

/* Number of FP32 entries of the parameter vector (complex entries count twice); -1 for NULL. */
int64_t ie_fno_param_count(const ie_fno* fno);

/* Issue all work on this CUDA stream (a cudaStream_t passed as void*; NULL = legacy default). */
ie_status ie_fno_set_stream(ie_fno* fno, void* stream);

/* Pointwise channel maps of the forward pass (the layers' v W + w, the head's Q1 and Q2) on the
 * fifth-generation tensor cores (on = 1, the default) or on the CUDA cores (0). The tensor-core path is
 * taken for BF16 storage when the map's input width is a multiple of 16 (at most 128) and its output
 * width at most 128: BF16 operands, FP32 accumulation in tensor memory (tcgen05.mma); its results agree
 * with the CUDA-core path to BF16 rounding. A kernel whose bounded wait for its MMAs gives up makes the
 * next forward call return IE_ECUDA. IE_EINVAL for another value of on. */
ie_status ie_fno_set_tensor_cores(ie_fno* fno, int32_t on);

/* Load (and reset the Adam state) / read back the parameter vector, host FP32, synchronous. */
ie_status ie_fno_set_params(ie_fno* fno, const float* host);
ie_status ie_fno_get_params(ie_fno* fno, float* host);

/* u = FNO(a) for batch samples: a_dev [batch][n^3][cin] FP32, u_dev [batch][n^3][cout] FP32 (device).
 * Keeps the activations that ie_fno_backward needs. */
ie_status ie_fno_forward(ie_fno* fno, int32_t batch, const float* a_dev, float* u_dev);

/* Gradient of a scalar loss with dL/du = du_dev ([batch][n^3][cout] FP32, device) with respect to every
 * parameter, for the activations of the preceding ie_fno_forward on the same a_dev and batch. The
 * gradient stays on the device for the optimiser; grads_host (may be NULL) receives a copy in the
 * parameter layout (synchronous). */
ie_status ie_fno_backward(ie_fno* fno, int32_t batch, const float* a_dev, const float* du_dev, float* grads_host);

/* One Adam step (beta 0.9, 0.999, eps 1e-8, step size lr) on the loss mean_b |u_b - t_b| / |t_b|
 * (relative L2 per sample). t_dev [batch][n^3][cout] FP32. loss (may be NULL) receives the loss before
 * the step (synchronous when non-NULL). */
ie_status ie_fno_train_step(ie_fno* fno, int32_t batch, const float* a_dev, const float* t_dev, float lr, float* loss);

/* Warm-start encoding (see above) of one sample. encode: a_dev [n^3][12] from sigma6_dev, the background
 * sigma0 and the right-hand side b_dev; writes |b| to bnorm_dev[0] (device double). encode_target:
 * t_dev [n^3][6] from the block solution E_dev. decode: x0_dev = b + |b|/sqrt(N) u (complex128 field)
 * from one sample's prediction u_dev [n^3][6]. */
ie_status ie_fno_encode(ie_fno* fno, const double* sigma6_dev, double sigma0, const double* b_dev, float* a_dev,
                        double* bnorm_dev);
ie_status ie_fno_encode_target(ie_fno* fno, const double* E_dev, const double* b_dev, const double* bnorm_dev,
                               float* t_dev);
ie_status ie_fno_decode(ie_fno* fno, const float* u_dev, const double* b_dev, const double* bnorm_dev, double* x0_dev);

/* Last error message (never NULL). */
const char* ie_fno_last_error(const ie_fno* fno);

/* Release the network and its device memory (synchronises its stream). NULL is allowed. */
void ie_fno_destroy(ie_fno* fno);

#ifdef __cplusplus
}
#endif
#endif /* IE_GB300_FNO_H */
