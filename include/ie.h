/*
 * ie.h — C ABI of the GB300 integral-equation (IE) forward model with domain decomposition.
 *
 * The library solves the discretised electric-field integral equation (eq. 8 of Saputera et al.,
 * "3D induction log modelling with integral equation method and domain decomposition
 * preconditioning"):
 *
 *     (I - G dsigma) E = E0,       dsigma = sigma - sigma0 I          (Section 2.1, eqs. 3, 8)
 *
 * on a uniform voxel grid embedded in a homogeneous isotropic background sigma0, for magnetic-dipole
 * transmitters, and returns the total magnetic field H = H0 + H^s at receivers (eq. 4). G is the
 * convolution with the electric Green's dyadic (eqs. 5, 7), evaluated with zero-padded 3D FFTs
 * (eq. 10); its singular cell is integrated over a sphere of equal volume (Section 2.2). The solve
 * is restarted GMRES (Section 2.2) inside the block Gauss-Seidel / block Jacobi sweeps of Algorithm 1
 * (Section 2.3, eqs. 21, 23) with the adaptive sub-domain tolerance e/10; sub-domains are slabs
 * along z (the tool axis). All compute runs in sm_103a CUDA kernels on the current device.
 *
 * Conventions
 *   - Time dependence e^{-i omega t}; mu = mu0; displacement currents ignored (Section 2.1).
 *   - Grid: nx*ny*nz cubic cells of edge h; cell (ix,iy,iz) has centre origin + (i + 1/2) h. Arrays
 *     over cells are x-fastest: index (iz*ny + iy)*nx + ix.
 *   - Complex arrays on the host are interleaved (re, im) doubles. Fields are component-major:
 *     [3][nz][ny][nx] complex.
 *   - sigma6: absolute conductivity per cell, [nz][ny][nx][6] doubles (xx, yy, zz, xy, xz, yz), S/m;
 *     the symmetric tensor must be positive definite (Appendix C tensors are).
 *   - A magnetic dipole of moment m (A m^2) is the magnetic current J^H = i omega mu0 m delta(r - r_s)
 *     in eq. 1, so H0 is the textbook dipole field.
 *   - Ownership: the caller owns every pointer it passes; the library copies inputs during the call
 *     and writes outputs before returning. Device memory used internally belongs to the context.
 *   - Errors: every call returns an ie_status; no exception crosses the ABI. ie_last_error() gives
 *     the context's last message. A failed call leaves the context usable unless it returns
 *     IE_ECUDA (a CUDA runtime error; the context should then be destroyed).
 *   - Threads: one context per host thread. Work is issued on the context's stream (default: the
 *     legacy default stream; see ie_set_stream) and every host-buffer call synchronises it.
 */
#ifndef IE_GB300_H
#define IE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IE_OK = 0,
  IE_EINVAL = 1,   /* invalid argument (sizes, NaN/indefinite sigma, source/receiver on a cell centre) */
  IE_ENOMEM = 2,   /* device or host allocation failed */
  IE_ECUDA = 3,    /* CUDA runtime error */
  IE_ENOCONV = 4,  /* iteration limit reached; outputs hold the best iterate, info is filled */
  IE_ESTATE = 5    /* call out of order (e.g. ie_solve before ie_set_contrast) */
} ie_status;

typedef enum { IE_DD_NONE = 0, IE_DD_JACOBI = 1, IE_DD_GAUSS_SEIDEL = 2 } ie_dd_mode;

typedef enum {
  IE_PREC_MIXED = 0, /* complex64 FFT convolution and Krylov vectors; FP64-accurate outer residual/refinement */
  IE_PREC_FP64 = 1,  /* complex128 everywhere */
  IE_PREC_DFLOAT = 2 /* ie_matvec only: the double-float (FP32-pair, ~46-bit) kernels of the outer residual */
} ie_precision;

typedef struct {
  int32_t nx, ny, nz;
  double origin[3]; /* minimum corner of the grid, metres */
} ie_grid;

typedef struct {
  double pos[3];    /* metres */
  double moment[3]; /* A m^2 */
} ie_dipole;

typedef struct {
  int32_t n_blocks;       /* number of sub-domains along z (>= 1); ignored for IE_DD_NONE */
  const int32_t* z_split; /* n_blocks+1 increasing z indices from 0 to nz, or NULL for equal slabs */
  int32_t restart;        /* GMRES restart length m (default 30) */
  int32_t max_outer;      /* maximum DD sweeps / refinement steps (default 50) */
  int32_t max_inner;      /* maximum GMRES iterations per block solve (default 20*restart) */
  int32_t precision;      /* ie_precision (default IE_PREC_MIXED) */
  int32_t adaptive;       /* 1: block tolerance e/10 (Algorithm 1, "-A"); 0: fixed_tol ("-F") */
  double fixed_tol;       /* block tolerance when adaptive == 0 */
  int32_t contraction;    /* 1: each block solve runs GMRES on the contraction form (see
                             ie_matvec_contraction); 0 (default): on the conventional operator */
  int32_t graph;          /* 1: each block solve is one CUDA graph (Givens rotations, stopping test
                             and restarts on the device, one host synchronisation per block solve;
                             per-kernel timing of ie_profile_enable then covers only the launches
                             outside the graph); 0 (default): host-driven Arnoldi loop */
  int32_t outer_krylov;   /* 1: flexible GMRES(outer_restart) on the whole-grid system, preconditioned by
                             one DD sweep (dd_mode) with block tolerance outer_inner_tol, instead of the
                             fixed-point sweeps of Algorithm 1 (the paper's conclusion); 0 (default) */
  int32_t outer_restart;  /* restart length of that outer iteration (default 10, at most 127) */
  double outer_inner_tol; /* block tolerance inside its preconditioner sweeps (default 0.1) */
  int32_t concurrent_blocks; /* 1 with IE_DD_JACOBI: the sub-domain solves of a sweep run at the same time,
                                each on its own stream and workspace (eq. 23 makes them independent; the
                                closing remark of Section 2.3 calls them parallelisable); their right-hand
                                sides and results are exchanged with the whole-grid field on the context
                                stream. Costs one Krylov basis per sub-domain. 0 (default): one after
                                another. Ignored for the other modes. */
} ie_opts;

#define IE_MAX_HISTORY 128
typedef struct {
  int32_t outer_iters;       /* DD sweeps (or refinement steps; with outer_krylov the preconditioner
                                sweeps) performed, summed over sources */
  int32_t gmres_iters_total; /* Arnoldi steps over all block solves and sources */
  int32_t matvecs;           /* block operator applications (Arnoldi + restart residuals) */
  int32_t n_history;         /* entries used in residual_history (first source only) */
  double final_rel_residual; /* max over sources of the FP64-accurate e (eq. 9) at exit, measured over
                                the sub-domains with contrast (the whole grid when all have some) */
  double seconds;            /* wall time of the call */
  double residual_history[IE_MAX_HISTORY]; /* e before the first sweep and after each sweep (with
                                              outer_krylov: the outer GMRES estimate after each step) */
  int32_t sweep_gmres_iters[IE_MAX_HISTORY]; /* GMRES iterations per sweep (first source) */
  int32_t reorth_passes;     /* Arnoldi steps that needed a second Gram-Schmidt pass */
  int32_t warm_start_used;   /* 1 if the guess of ie_set_initial_field_dev replaced E := E0 */
  double cold_rel_residual;  /* with a guess given: e (eq. 9) of E = E0 and of the guess; else 0 */
  double warm_rel_residual;
  int32_t active_blocks;     /* sub-domains with contrast, summed over sources: only these are swept and
                                e is measured over them (Section 3.1); the field of the others is
                                E0 + G dsigma E from the final residual */
} ie_info;

typedef struct ie_ctx ie_ctx;

/* Default options (restart 30, max_outer 50, max_inner 600, mixed precision, adaptive). */
void ie_default_opts(ie_opts* opts);

/* Create a context for one grid, cell size h (m), background sigma0 (S/m) and frequency (Hz)
 * (Section 2.1: homogeneous isotropic background; eq. 7: k0 = sqrt(i omega mu0 sigma0)). Tabulates
 * the Green kernel in FP64 (eq. 5 plus the equal-volume-sphere self term of Section 2.2), takes its
 * FFT (eq. 10, padding to the next power of two >= 2n per axis, at most 1024) and stores one octant
 * of the six symmetric components in complex128 and complex64. Requires 1 <= nx, ny, nz <= 512.
 * Returns IE_EINVAL for bad sizes or non-positive h, sigma0, freq. *out is NULL on failure. */
ie_status ie_create(const ie_grid* grid, double cell_size_m, double sigma0_S_per_m, double freq_hz, ie_ctx** out);

/* Issue all work on this CUDA stream (a cudaStream_t passed as void*; NULL = legacy default). */
ie_status ie_set_stream(ie_ctx* ctx, void* cuda_stream);

/* Set the conductivity model from a host array sigma6 [nz][ny][nx][6] (see Conventions); forms the
 * contrast dsigma = sigma - sigma0 I (Section 2.1). IE_EINVAL if any value is not finite or a tensor
 * is not positive definite (the previous model is then kept only if the call fails before upload). */
ie_status ie_set_contrast(ie_ctx* ctx, const double* sigma6);
/* Same, from a device array with the same layout. */
ie_status ie_set_contrast_dev(ie_ctx* ctx, const double* sigma6_dev);

/* Forward model for n_src transmitters and n_rx receivers (Algorithm 1 and eq. 4).
 *   dd_mode IE_DD_NONE: one GMRES on the whole grid (Section 2.2);
 *           IE_DD_GAUSS_SEIDEL / IE_DD_JACOBI: Algorithm 1 with opts->n_blocks slabs along z.
 *   tol: target whole-domain relative residual e (eq. 9), verified in FP64.
 *   rx_xyz: [n_rx][3] receiver positions; H_out: [n_src][n_rx][3] complex (interleaved), total H.
 *   opts and info may be NULL. Sources/receivers closer than 1e-9 h to a cell centre -> IE_EINVAL.
 * Returns IE_ENOCONV (with H_out and info written for the best iterate) when max_outer sweeps or the
 * inner iteration limits end before e <= tol. */
ie_status ie_solve(ie_ctx* ctx, int32_t n_src, const ie_dipole* src, int32_t n_rx, const double* rx_xyz,
                   int32_t dd_mode, double tol, const ie_opts* opts, double* H_out, ie_info* info);

/* One forward problem of a batch: inputs as for ie_solve, outputs written by ie_solve_batch. */
typedef struct {
  ie_ctx* ctx;             /* context of the item (grid, cell size, background, frequency, contrast) */
  const double* sigma6;    /* host [nz][ny][nx][6] conductivity set before the solve, or NULL to keep
                              the context's current model */
  int32_t n_src;
  const ie_dipole* src;
  int32_t n_rx;
  const double* rx_xyz;    /* [n_rx][3] */
  int32_t dd_mode;
  double tol;
  const ie_opts* opts;     /* may be NULL */
  double* H_out;           /* [n_src][n_rx][3] complex */
  ie_info* info;           /* may be NULL */
  ie_status status;        /* result of this item */
  const double* E_init_dev; /* may be NULL: initial guess for this item's first source, as for
                               ie_set_initial_field_dev (device complex128 [3][nz][ny][nx]) */
} ie_batch_item;

/* Many independent forward problems (tool positions x frequencies, Section 3.3's moving window) in
 * flight together. Items that share a context run one after another in the given order; different
 * contexts run concurrently, each on its own CUDA stream driven by one of up to max_concurrent host
 * threads (0: one per distinct context, at most 16), so their kernels overlap on the GPU. A context
 * still on the legacy default stream gets a private non-blocking stream for the call. Every item's
 * status is written; the call returns IE_OK if all items did, else the first non-OK status in item
 * order. An item without sigma6 uses the contrast already set on its context. */
ie_status ie_solve_batch(int32_t n_items, ie_batch_item* items, int32_t max_concurrent);

/* Copy the electric field of the last source of the last ie_solve to the host ([3][nz][ny][nx]
 * complex, interleaved). IE_ESTATE if no solve has run. */
ie_status ie_get_field(ie_ctx* ctx, double* E_out);

/* The contraction form of one sub-domain's operator (the remedy for high contrast named at the end of
 * Section 2.3): y = (M - G^(ii) dsigma^(i) M) x with M = 2 sigma0 (sigma + sigma0 I)^-1 per voxel, i.e.
 * the operator of ie_matvec right-multiplied by M. M - G dsigma M = I - C r with C = I + 2 sigma0 G and
 * r = (sigma - sigma0 I)(sigma + sigma0 I)^-1, a contraction for a positive definite sigma, so GMRES
 * converges in fewer iterations at high contrast. A solve with ie_opts.contraction = 1 finds u with
 * (M - G dsigma M) u = b and adds M u to the field: the residual, its norm and the stopping rule are those
 * of the conventional system. Same arguments, layouts and precisions (MIXED, FP64) as ie_matvec. */
ie_status ie_matvec_contraction(ie_ctx* ctx, int32_t precision, int32_t z0, int32_t nz, const double* x, double* y);

/* Device-pointer variants (no synchronisation; complex128 [3][nz][ny][nx] on the current device):
 * copy the field of the last solve into E_dev (IE_ESTATE if none), or write the incident field of one
 * dipole into E0_dev. */
ie_status ie_get_field_dev(ie_ctx* ctx, double* E_dev);
ie_status ie_incident_field_dev(ie_ctx* ctx, const ie_dipole* src, double* E0_dev);

/* Initial guess for the next ie_solve (its first source): E_dev, complex128 [3][nz][ny][nx] on the
 * device, is copied on the context stream and replaces the initial E := E0 of Algorithm 1 if its FP64
 * residual e (eq. 9) is smaller than that of E0; otherwise the solve starts from E0 as usual (ie_info
 * reports both residuals and the choice). The guess is consumed by that solve. NULL clears it. */
ie_status ie_set_initial_field_dev(ie_ctx* ctx, const double* E_dev);

/* Apply the operator of one sub-domain, y = (I - G^(ii) dsigma^(i)) x (eq. 8 restricted to the slab
 * z in [z0, z0+nz), block-sized FFT convolution as used inside GMRES), on host arrays
 * x, y: [3][nz][ny][nx] complex. precision selects the complex64 or complex128 kernels. */
ie_status ie_matvec(ie_ctx* ctx, int32_t precision, int32_t z0, int32_t nz, const double* x, double* y);

/* The same complex64 operator on device arrays (x_dev, y_dev: [3][nz][ny][nx] float2, distinct),
 * enqueued on the context stream without synchronising. */
ie_status ie_matvec_dev(ie_ctx* ctx, int32_t z0, int32_t nz, const void* x_dev, void* y_dev);

/* Same operator as ie_matvec_dev, for callers that must not allocate device memory during the call.
 * (An extension of this library; the paper has no counterpart.) Who needs it: a host application that
 * hands the library a fixed device-memory budget (its own pool owns the rest of the GPU, so a
 * cudaMalloc inside the call could fail with out-of-memory at an arbitrary point), and latency-bound
 * loops that cannot afford cudaMalloc/cudaFree, which may synchronise the whole device and stall the
 * caller's other streams. The FFT intermediates go to one fixed 16 MiB device array that the library
 * holds on every GPU that loads it, until the process exits: the x-transformed slab A
 * (8 * 3 * nz * ny * Lx bytes), padded up to a 256-byte boundary, then the xy-transformed slab B
 * (8 * 3 * nz * Ly * Lx bytes), with Lx/Ly the padded FFT lengths; a slab whose A and B do not fit is
 * rejected with IE_EINVAL and nothing is enqueued. The Green spectra for the slab height must already
 * exist (ie_create prepares the whole grid; other heights are prepared by one ie_matvec_dev or ie_solve
 * call first), else IE_ESTATE. The passes use the default FFT tile shapes (the autotuner is not
 * consulted, since timing candidates would need scratch of its own). The first call on each device
 * looks up the array's device address on that device (the call runs on the context's device); make
 * that first call before any stream capture. All calls share the array and it keeps the last call's
 * contents: every element a call reads was written earlier in the same call, so nothing needs
 * clearing, but calls that overlap on the GPU (different streams or contexts at the same time) race
 * and give wrong results. x_dev, y_dev: distinct device arrays [3][nz][ny][nx] complex64; work is
 * enqueued on the context stream without synchronising. */
ie_status ie_matvec_dev_noalloc(ie_ctx* ctx, int32_t z0, int32_t nz, const void* x_dev, void* y_dev);

/* Interaction field of eqs. 21/23: y = G^(ts) dsigma^(s) x for a source slab [zs0, zs0+nzs) and a
 * target slab [zt0, zt0+nzt), computed with the whole-grid spectra (complex128 kernels). x: source
 * field [3][nzs][ny][nx], y: target field [3][nzt][ny][nx], host, complex. */
ie_status ie_interaction(ie_ctx* ctx, int32_t zs0, int32_t nzs, int32_t zt0, int32_t nzt, const double* x, double* y);

/* Restarted GMRES (Section 2.2) on one sub-domain operator (slab [z0, z0+nz)): solves
 * (I - G^(ii) dsigma^(i)) x = b from x0 (NULL = 0) to ||b - A x|| <= tol ||b||, host arrays.
 * iters and rel_res (true final residual) may be NULL. IE_ENOCONV when max_iter is reached. */
ie_status ie_gmres(ie_ctx* ctx, int32_t precision, int32_t z0, int32_t nz, const double* b, const double* x0,
                   double tol, int32_t restart, int32_t max_iter, double* x, int32_t* iters, double* rel_res);

/* Green spectra for a slab of nz_set cells (nz_set = a sub-domain's nz, or the grid nz for the
 * interaction spectra): component comp (0 xx, 1 yy, 2 zz, 3 xy, 4 xz, 5 yz) of the octant
 * F[K](kx, ky, kz) / (Lx Ly Lz) for 0 <= k <= L/2 per axis, complex128, layout [kz][ky][kx].
 * dims_out (may be NULL) receives (Lx, Ly, Lz). */
ie_status ie_green_spectrum(ie_ctx* ctx, int32_t nz_set, int32_t comp, double* out, int32_t* dims_out);

/* Incident electric field E0 of one dipole on the cell centres, [3][nz][ny][nx] complex (host). */
ie_status ie_incident_field(ie_ctx* ctx, const ie_dipole* src, double* E0_out);

/* Total magnetic field at receivers for a given electric field E ([3][nz][ny][nx] complex, host):
 * H = H0 + sum_j dv grad g(r - r_j) x (dsigma_j E_j) (eqs. 4, 6). H_out [n_rx][3] complex. */
ie_status ie_receiver_fields(ie_ctx* ctx, const double* E, const ie_dipole* src, int32_t n_rx, const double* rx_xyz,
                             double* H_out);

/* Padded FFT lengths (Lx, Ly, Lz) the context uses for a slab of nz_set cells. */
ie_status ie_fft_dims(const ie_ctx* ctx, int32_t nz_set, int32_t* dims_out);

/* Kernel classes for the built-in launch accounting (see ie_profile_enable). */
typedef enum {
  IE_K_P1_C64 = 0,  /* contrast product + x-FFT (complex64) */
  IE_K_P2_C64 = 1,  /* y-FFT (complex64) */
  IE_K_P3_C64 = 2,  /* z-FFT + Green product + inverse z-FFT (complex64) */
  IE_K_P4_C64 = 3,  /* inverse y-FFT (complex64) */
  IE_K_P5_C64 = 4,  /* inverse x-FFT + crop + combine (complex64) */
  IE_K_P1_C128 = 5, IE_K_P2_C128 = 6, IE_K_P3_C128 = 7, IE_K_P4_C128 = 8, IE_K_P5_C128 = 9,
  IE_K_DOTS = 10,        /* Arnoldi inner products */
  IE_K_UPDATE = 11,      /* Arnoldi vector updates */
  IE_K_KRYLOV_MISC = 12, /* reductions, scaling, basis combination, norms */
  IE_K_FIELD = 13,       /* incident field, receivers, contrast, field copies */
  IE_K_SETUP = 14,       /* Green tabulation and spectra */
  IE_K_COUNT = 15
} ie_kernel_class;

/* Launch accounting. Every kernel launch is always counted per class together with its algorithmic
 * bytes (the HBM bytes the pass model says it must move). With on != 0, each launch is also
 * bracketed by CUDA events on the context stream and its device time accumulated. Resets counters. */
ie_status ie_profile_enable(ie_ctx* ctx, int32_t on);
/* Counters of one class since the last ie_profile_enable: launches, device milliseconds (0 unless
 * timing was on) and algorithmic bytes. Any output pointer may be NULL. */
ie_status ie_profile_read(const ie_ctx* ctx, int32_t kclass, int64_t* launches, double* ms, double* algo_bytes);

/* Tile shapes chosen so far by the FFT-tile autotuner of this process, as text (one line per pass
 * shape: pass, element bytes, pencil length, Lx, Ly, slab heights, chosen variant, then the measured
 * microseconds per launch of every variant). Variants 0/1/2 of the y passes and 0/1/4/6 of the z pass
 * are tiles of about 256 (z: 128), half, twice (and z: four times) as many threads; z-pass variants
 * 2/3/5/7 are the same four with TMA staging of their input; z-pass variants 8/9 (256 threads) and
 * 10/11 (512 threads) pair each row ky with its mirror Ly - ky, without and with TMA staging.
 * Writes at most len bytes including the terminating NUL; returns the length the full text needs. */
int32_t ie_tuned_tiles(char* buf, int32_t len);

/* Testing hook (an extension of this library; the paper has no counterpart): after `after` more
 * successful device allocations, the next one made by any context of this process reports
 * out-of-memory without calling cudaMalloc, so callers can test their handling of IE_ENOMEM without
 * exhausting a GPU. Fires once; a negative value switches it off. The call that meets the injected
 * failure returns IE_ENOMEM and leaves its context usable (nothing half-allocated is kept). */
void ie_debug_fail_allocation(int32_t after);

/* Testing hook (an extension of this library; the paper has no counterpart): every later convolution of
 * this process runs pass `pass` (2 = the y pass P2, 3 = the z pass P3, 4 = the inverse y pass P4) in
 * tile variant `variant` (the numbering of ie_tuned_tiles) instead of the autotuned one; -1 returns the
 * pass to the autotuner. All variants compute bit-identical results, and this hook lets a test check
 * that. A z-pass variant that the arithmetic in use does not build (8 and 9 outside complex64) makes the
 * convolution fail with IE_ECUDA. IE_EINVAL for a pass or variant out of range. The setting is a
 * process-wide atomic; a convolution that another thread is already enqueuing may still use the
 * previous choice. */
ie_status ie_debug_force_tile(int32_t pass, int32_t variant);

/* Last error message of the context (never NULL; "" when none). */
const char* ie_last_error(const ie_ctx* ctx);

/* Release the context and all its device memory. NULL is allowed. */
void ie_destroy(ie_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* IE_GB300_H */
