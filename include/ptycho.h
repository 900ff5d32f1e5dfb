/*
 * ptycho.h - C ABI of the GB300 multi-wavelength, multi-mode ptychography hot path.
 *
 * The library evaluates the universal ptychography model of arXiv 2311.14780, Eq. 1,
 *
 *   I_j = M[ sum_l sum_m | D_{lambda_l,z}[ sigma_j P_lm(r) O_l(r - s_j) ] |^2 + N ],
 *
 * written as the composite f5(f4(f3(f1(sigma_j), f2(s_j)))) of Eq. 2, scores it with the
 * amplitude (MSE on the modulus) or Poisson loss of the section "Universal Ptychography
 * Algorithm based on Automatic Differentiation", returns the analytic gradient that the
 * paper obtains by reverse-mode differentiation (Fig. 1B), and applies Adam.  One sample
 * mode per wavelength (N = 1 in Eq. 1), as in the paper's reconstructions.
 *
 * Conventions shared by every entry point
 *   - Complex arrays are complex64: interleaved (re, im) float pairs, row-major.
 *   - Array arguments of compute calls are DEVICE pointers owned by the caller.  The
 *     library never frees them and only reads inputs / overwrites outputs.
 *   - Objects of all wavelengths are packed into one buffer: O_l starts at complex offset
 *     sum_{l' < l} obj_h[l'] * obj_w[l'] and is obj_h[l] x obj_w[l] row-major.
 *   - Probes: P[L][M][F][F].  Predicted / measured patterns: [J][F][F] float, camera grid,
 *     zero frequency at (F/2, F/2).
 *   - Propagation D is the orthonormal 2D DFT with the zero frequency moved to the centre;
 *     each wavelength is sampled at its own object pixel size (lambda_l z / (F p)), so all
 *     wavelengths share one detector grid.
 *   - Gradients use g = dL/dRe + i dL/dIm for every complex parameter.
 *   - Compute calls are asynchronous on ``stream`` (a cudaStream_t passed as void*; NULL =
 *     the legacy default stream) and must be issued on the device that was current when
 *     the plan was created.  Calls on one plan share its workspace: do not run two calls
 *     of the same plan concurrently on different streams.
 *   - Return value: 0 on success, a negative PTYCHO_E* code otherwise (text through
 *     ptycho_strerror).  Argument errors are detected on the host before any launch.
 */
#ifndef PTYCHO_GB300_H
#define PTYCHO_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PTYCHO_OK 0
#define PTYCHO_EINVAL (-1)       /* bad shape, size, NULL pointer or option            */
#define PTYCHO_ERANGE (-2)       /* a scan position puts a patch outside its object   */
#define PTYCHO_ENOMEM (-3)       /* device allocation of the plan workspace failed     */
#define PTYCHO_ECUDA (-4)        /* a CUDA call or kernel launch failed                */
#define PTYCHO_ETIMEDOUT (-5)    /* a bounded device wait ran out (serving loop)       */
#define PTYCHO_EUNSUPPORTED (-6) /* frame size not in {64, 128, 256, 512}, L > 16      */
#define PTYCHO_ETOOLARGE (-7)    /* problem does not fit ptycho_forward_noalloc's array */
#define PTYCHO_EBUSY (-8)        /* serving: no free slot, or the HBM budget is exhausted  */

/* Pipeline variants (ptycho_geom_t.flags).  All give the same results up to FP32 rounding.
 * RECOMPUTE_COLUMNS: the adjoint recomputes the column DFT from the kept row-pass output
 *   instead of keeping Psi (less memory traffic, one more 1D pass per evaluation); the
 *   default for F >= 256, where it measured faster.
 * KEEP_PSI: keep Psi between the passes (the default for F < 256).
 * OBJ_GRAD_ATOMIC: the row adjoint adds the object gradient with FP32 atomics instead of
 *   the tile-owned gather (faster; the summation order, and so the last bits of grad O,
 *   then vary between runs).
 * TMA / NO_TMA: the column passes stage each mode's column block in shared memory with
 *   bulk tensor copies (TMA) / read S with ordinary loads.  Default: TMA for F >= 512, and
 *   for F = 128 when a position has at least four fields (L*M >= 4), where it measured
 *   faster; otherwise the larger shared-memory footprint costs more occupancy than the
 *   copies save.  NO_TMA wins when both are given.
 * UNFUSED_ROW_ADJ / FUSED_ROW_ADJ: one block of the adjoint row pass per probe mode, each mode's
 *   object-gradient row left in the scratch for the object-gradient kernel / all modes of a
 *   wavelength per block, the probe rows read once per batch and the object-gradient rows summed
 *   over the modes before they are written.  The fused pass needs all modes of a position in the
 *   scratch and T*M <= 256 (T = 4, 8, 16, 16 threads per row for F = 64, 128, 256, 512; 32 with
 *   one warp per row).  Default: fused for F <= 256; at F = 512 fused from 2 modes up where the
 *   one-warp rows fit (M <= 10), and from 8 modes up otherwise; per mode with one mode (measured
 *   5-9 % faster there).  UNFUSED_ROW_ADJ wins when both are given.
 * STAGED_COLUMNS: whenever all modes of a position fit the scratch, run each column block over
 *   all modes of W columns of one position, copying the next mode's columns into shared memory
 *   (cp.async, double-buffered) while the current one is transformed (one intensity slice, no
 *   mode groups).  Measured slower than the default mode groups on every benchmark workload
 *   (fewer warps per SM); NARROW_COLUMNS takes 4 columns per block instead of 8.
 * FUSED_ROW_FWD / UNFUSED_ROW_FWD: the forward row pass over all modes of a wavelength per
 *   block, the probe row in registers and the next position's object rows prefetched
 *   (cp.async) / one block per position and row block.  Default: fused at F = 512 from 4 modes
 *   (the probes outgrow the L2 there; measured 2-3 % faster), per position otherwise (measured
 *   faster with one mode and at 256^2).  UNFUSED_ROW_FWD wins when both are given.
 * NO_PDL: launch without programmatic dependent launch.
 * ROWS_16_THREADS: at F = 512 the fused row adjoint takes one warp per row (16 values per lane,
 *   probe rows through L1/L2, two blocks of at most 320 threads per SM) whenever 32*M*rpb <= 320:
 *   measured 6 % faster on 512^2 x 10 modes x 6 wavelengths than 16 threads per row.  This flag
 *   keeps 16 threads per row in both fused row passes (so do ROW_ADJ_PROBE_L2 and
 *   ROW_ADJ_PROBE_SMEM for the adjoint).
 * COLS_ONE_BLOCK: at F = 512 the TMA-staged column passes (without KEEP_PSI) transpose in two
 *   halves through an exchange area of half the size and the adjoint reads its dL/dI factors
 *   through L1/L2, so two blocks fit on an SM (99 KB of shared memory each); this flag keeps the
 *   one-block passes (full exchange, staged factors).
 * FWD_ROWS_WARP: at F = 512 the fused forward row pass with one warp per row as well (when
 *   32*M*rpb <= 320).  Measured 1.7 % slower per step on 512^2 x 10 modes x 6 wavelengths (146.4
 *   vs 144.0 ms): its twice as many resident warps take the SMs from the other streams' passes.
 * ROW_ADJ_PROBE_L2 / ROW_ADJ_PROBE_SMEM: the fused row adjoint with T threads per row reads its
 *   probe rows through L1/L2 (and is compiled for two blocks of at most 160 threads per SM) /
 *   holds them in shared memory for the batch.  Default below F = 512: shared memory; at F = 512
 *   where the one-warp rows do not fit, L1/L2 when T*M*rpb <= 160.  PROBE_SMEM wins when both are
 *   given.
 * RESIDENT_FRAMES: at F <= 128, frame-resident passes instead of the scratch passes: one
 *   block holds a whole F x F field in shared memory, so exit waves and spectra never leave
 *   the SM; the forward writes only the per-position intensity, the adjoint recomputes Psi on
 *   chip and writes only each mode's object-gradient patch.  Measured 0.5-0.9x the speed of
 *   the default scratch passes (the transforms are bound by the shared-memory pipe either way,
 *   and a 128^2 frame leaves room for one block of 16 warps per SM; the adjoint recomputes Psi).
 *   Ignored at F >= 256, with registered offsets, with the chirp-z propagator, with modes in
 *   chunks, and with OBJ_GRAD_ATOMIC. */
#define PTYCHO_FLAG_RECOMPUTE_COLUMNS 1
#define PTYCHO_FLAG_OBJ_GRAD_ATOMIC 2
#define PTYCHO_FLAG_KEEP_PSI 4
#define PTYCHO_FLAG_NO_TMA 8
#define PTYCHO_FLAG_TMA 16
#define PTYCHO_FLAG_UNFUSED_ROW_ADJ 32
#define PTYCHO_FLAG_STAGED_COLUMNS 64
#define PTYCHO_FLAG_NARROW_COLUMNS 128
#define PTYCHO_FLAG_FUSED_ROW_FWD 256
#define PTYCHO_FLAG_NO_PDL 512
#define PTYCHO_FLAG_RESIDENT_FRAMES 1024
#define PTYCHO_FLAG_ROW_ADJ_PROBE_L2 2048
#define PTYCHO_FLAG_ROW_ADJ_PROBE_SMEM 4096
#define PTYCHO_FLAG_UNFUSED_ROW_FWD 8192
#define PTYCHO_FLAG_ROWS_16_THREADS 16384
#define PTYCHO_FLAG_FWD_ROWS_WARP 32768
#define PTYCHO_FLAG_COLS_ONE_BLOCK 65536
#define PTYCHO_FLAG_FUSED_ROW_ADJ 131072

#define PTYCHO_LOSS_AMPLITUDE 0  /* sum (sqrt(I + eps) - sqrt(Ihat))^2                  */
#define PTYCHO_LOSS_POISSON 1    /* sum (I + eps) - Ihat - Ihat log((I + eps) / Ihat)   */
/* Mixed Poisson-Gaussian noise (the paper's MLE with mixed statistics), shifted-Poisson
 * reading: the Poisson deviance of (I + eps + s2, max(Ihat + s2, 0)), s2 = read_noise_var. */
#define PTYCHO_LOSS_POISSON_GAUSSIAN 2

typedef struct ptycho_plan ptycho_plan_t;

/* Problem description (all pointers are HOST pointers, read during ptycho_plan_create). */
typedef struct {
  int32_t L;                /* wavelengths (Eq. 1 index l), 1..16                       */
  int32_t M;                /* incoherent probe modes per wavelength (index m), >= 1    */
  int32_t F;                /* frame side: 64, 128, 256 or 512                          */
  int32_t J;                /* scan positions (the paper's index k), >= 1               */
  const int32_t* obj_h;     /* [L] object rows, >= F                                    */
  const int32_t* obj_w;     /* [L] object columns, >= F                                 */
  const int32_t* pos;       /* [L][J][2] (row, col) of each patch's top-left corner in
                               wavelength-l object pixels: the integer scan shift s_j of
                               f2 (Eq. 2).  0 <= row <= obj_h[l] - F, same for col.
                               Bound at plan creation: a new scan needs a new plan.    */
  const double* lambda;     /* [L] wavelengths in metres (recorded; may be NULL)        */
  double z;                 /* sample-camera distance, metres (88 mm in the paper)      */
  double det_pixel;         /* camera pixel pitch, metres (15 um)                       */
  double tilt_rad;          /* angle of incidence from the surface normal (70 degrees)  */
  int32_t remap;            /* 1: apply the tilted-plane remap inside f5; 0: identity   */
  int32_t loss;             /* PTYCHO_LOSS_AMPLITUDE, _POISSON or _POISSON_GAUSSIAN     */
  float eps;                /* intensity floor added to I in the loss and its gradient  */
  int64_t scratch_bytes;    /* FFT scratch budget in bytes; 0 = library default (about
                               1200 evaluations but at least 64 positions per batch, at
                               least three batches per call, batches of equal size within
                               one position, at most 8 GiB per buffer set)              */
  int32_t overlap;          /* position batches in flight on separate streams (1..4), each
                               with its own scratch set; 0 = library default (3)       */
  int32_t flags;            /* PTYCHO_FLAG_* variants; 0 = defaults                      */
  int32_t col_groups;       /* mode groups of the column passes (partial intensity sums
                               per position); 0 = library default                       */
  float read_noise_var;     /* Gaussian read-noise variance s2 (photons^2, >= 0) of
                               PTYCHO_LOSS_POISSON_GAUSSIAN; ignored by the other losses */
  const double* zoom;       /* [L] or NULL.  Non-NULL selects the chirp-z propagator (the
                               paper's, Section "Benchmarking ..."): per wavelength the zoom
                               DFT Z[k'][n'] = exp(-2 pi i zoom[l] n' k' / F), centred
                               indices, Psi = (1/F) Z psi Z^T; zoom[l] = lambda_ref /
                               lambda_l puts every wavelength on one object grid (then
                               obj shapes and positions can be equal for all l).  Needs
                               all modes of a position in the scratch and no registered
                               offsets (PTYCHO_EUNSUPPORTED otherwise); 0 < zoom[l] <= 4.  NULL:
                               the orthonormal DFT with the DC at F/2.                  */
} ptycho_geom_t;

/* Adam state (Kingma & Ba), cited by the paper as its optimiser.  Real and imaginary
 * parts are separate real parameters.  m and v are DEVICE arrays with the layout of the
 * parameter they belong to (2 floats per complex element), zero-initialised by the caller. */
typedef struct {
  float lr_O, lr_P;         /* step sizes of the objects and of the probes              */
  float beta1, beta2, eps;  /* 0.9, 0.999, 1e-8 are the usual values                    */
  int32_t t;                /* steps taken so far; ptycho_step increments it            */
  float* mO; float* vO;     /* [2 * numel(O)]                                           */
  float* mP; float* vP;     /* [2 * numel(P)]                                           */
  int32_t* t_dev;           /* optional DEVICE step counter (zero-initialised): when set,
                               ptycho_step increments it on the device and the bias
                               correction reads it there, so a captured CUDA graph of
                               ptycho_step can be replayed; t is then left unchanged  */
  /* Optional: the power coefficients sigma and the background N are optimised too (the
   * paper lists both among the variables it reconstructs, and initialises them to 1). */
  float lr_sigma;           /* > 0: ptycho_step updates sigma [J] in place              */
  float lr_bg;              /* > 0: ptycho_step updates bg [F][F] in place              */
  float* m_sigma; float* v_sigma;   /* [J], required when lr_sigma > 0                  */
  float* m_bg; float* v_bg;         /* [F*F], required when lr_bg > 0                   */
  /* Optional: the fractional scan offsets registered with ptycho_plan_set_offsets are
   * optimised too (the paper refines the scan positions s_k with the other variables). */
  float lr_delta;                   /* > 0: ptycho_step updates the offsets in place          */
  float* m_delta; float* v_delta;   /* [L*J*2], required when lr_delta > 0                    */
  /* Optional: non-NULL (device, 1 double) makes ptycho_step also write dL/dz of its pass
   * (see g_z of ptycho_adjoint_ex; requires the remap).  z itself lives in the plan's host
   * geometry: the caller updates it with ptycho_plan_set_distance. */
  double* g_z;
  /* Optional object regularisation (see ptycho_regularise): reg_l1 > 0 or reg_tv > 0 adds the
   * regulariser with smoothing reg_eta (> 0) to the loss and its gradient to the object's
   * before Adam. */
  float reg_l1, reg_tv, reg_eta;
} ptycho_adam_t;

/* Validates the geometry and every scan position (PTYCHO_ERANGE names an out-of-object
 * patch: no wrap-around, no clamping), builds the remap operator R (bilinear, four taps
 * per camera pixel; camera pixels whose taps leave the model grid are masked) and its
 * exact transpose, the twiddle table, and allocates the device workspace.  The plan owns
 * everything it allocates.  Returns PTYCHO_ENOMEM if the workspace cannot be allocated. */
int ptycho_plan_create(const ptycho_geom_t* geom, ptycho_plan_t** out);

/* Frees the plan and its workspace (synchronises the device first).  NULL is accepted. */
int ptycho_plan_destroy(ptycho_plan_t* plan);

/* Bytes of device memory owned by the plan; complex element counts of O and P. */
int64_t ptycho_plan_workspace_bytes(const ptycho_plan_t* plan);
int64_t ptycho_plan_numel_O(const ptycho_plan_t* plan);
int64_t ptycho_plan_numel_P(const ptycho_plan_t* plan);

/* Forward model, Eq. 1 / Eq. 2: I_pred[j] for every scan position j.
 *   O      packed objects (complex64)           P    [L][M][F][F] complex64
 *   sigma  [J] power coefficients of f1, or NULL (all 1)
 *   bg     [F][F] background N on the model grid (added before the remap), or NULL
 *   I_pred [J][F][F] out: camera-grid prediction; pixels the remap cannot reach are 0 */
int ptycho_forward(ptycho_plan_t* plan, const float* O, const float* P, const float* sigma,
                   const float* bg, float* I_pred, void* stream);

/* Loss of the selected positions (section "Universal Ptychography Algorithm"):
 *   I_meas    [J][F][F] measured patterns (camera grid)
 *   mask      NULL (all pixels), [F][F] (mask_per_frame = 0) or [J][F][F] (= 1); nonzero
 *             = used.  Pixels the remap cannot reach are excluded in addition.
 *   batch_idx DEVICE int32 list of positions to include, or NULL for all J in order
 *   nbatch    entries of batch_idx (ignored when batch_idx is NULL)
 *   loss_dev  DEVICE double, out: sum over positions and used pixels (FP64 reduction) */
int ptycho_loss(ptycho_plan_t* plan, const float* O, const float* P, const float* sigma,
                const float* bg, const float* I_meas, const uint8_t* mask, int mask_per_frame,
                const int32_t* batch_idx, int nbatch, double* loss_dev, void* stream);

/* Loss and its gradient with respect to every O_l and P_lm (the reverse pass of Fig. 1B),
 * summed over the selected positions.  gO (numel(O) complex) and gP (numel(P) complex)
 * are OVERWRITTEN.  The propagated fields are kept in the plan's scratch between the
 * forward and adjoint passes when they fit its budget, and recomputed otherwise.
 * Arguments as for ptycho_loss; loss_dev may be NULL. */
int ptycho_adjoint(ptycho_plan_t* plan, const float* O, const float* P, const float* sigma,
                   const float* bg, const float* I_meas, const uint8_t* mask, int mask_per_frame,
                   const int32_t* batch_idx, int nbatch, float* gO, float* gP, double* loss_dev,
                   void* stream);

/* ptycho_adjoint that also returns the gradients with respect to the power coefficients,
 * the background and the fractional scan offsets (the paper's sigma_k, N(rho) and s_k,
 * Eq. 1), each optional (NULL = not computed):
 *   g_sigma [J] OVERWRITTEN: dL/dsigma_j for every position in the call, 0 for the others.
 *           Computed from the intensities: sigma_j enters every exit wave of frame j as a
 *           real factor and the DFT is unitary, so dL/dsigma_j = (2 / sigma_j) times the
 *           sum over the camera grid of (mask dL/dI) * (R sum_lm |Psi_jlm|^2); 0 where
 *           sigma_j = 0 (the derivative vanishes there).  sigma NULL means all ones.
 *   g_bg    [F][F] OVERWRITTEN: dL/dN on the model grid (N is added before the remap),
 *           the sum over the call's positions of R^T(mask dL/dI); deterministic for a
 *           given plan (per-stream partial sums added in a fixed order).
 *   g_delta [L][J][2] OVERWRITTEN: dL/ddelta[l][j] (rows, columns) for the positions in the
 *           call, 0 for the others; requires offsets registered with
 *           ptycho_plan_set_offsets (PTYCHO_EINVAL otherwise).  Computed in the Fourier
 *           domain: (1/F^2) Re sum_k conj(Ghat(k)) 2 pi i f(k) Q(k), Ghat the DFT of the
 *           gradient with respect to the shifted patch, Q the ramp times the DFT of the
 *           integer window, f in cycles per pixel.
 *   g_z     [1] (device, FP64) OVERWRITTEN: dL/dz, the derivative with respect to the
 *           propagation distance (a variable the paper optimises) at fixed object pixels and
 *           positions.  The propagator here is the orthonormal DFT, so z enters through the
 *           tilted-plane remap: dL/dz = sum over the call's frames and camera pixels of
 *           (mask dL/dI) * (s_row drow/dz + s_col dcol/dz), s the slopes of the bilinear
 *           interpolant of the model intensity (field + background) and (row, col) the
 *           pixel's fractional model-grid index; pixels whose taps leave the grid are held
 *           masked.  A caller with physical scan positions adds the chain through the object
 *           pixel size lambda z / (F p): sum over (l, j) of g_delta . d pos / dz.  Requires
 *           the remap (PTYCHO_EINVAL otherwise).
 * Other arguments as for ptycho_adjoint. */
int ptycho_adjoint_ex(ptycho_plan_t* plan, const float* O, const float* P, const float* sigma,
                      const float* bg, const float* I_meas, const uint8_t* mask, int mask_per_frame,
                      const int32_t* batch_idx, int nbatch, float* gO, float* gP, float* g_sigma,
                      float* g_bg, float* g_delta, double* g_z, double* loss_dev, void* stream);

/* Moves the camera to distance z (> 0, metres): rebuilds the plan's tilted-plane remap (taps,
 * their z rates and the transpose), for z correction driven by g_z.  Waits for the device
 * to be idle first (no call of this plan may be in flight) and is synchronous; may
 * reallocate the transpose's arrays.  PTYCHO_EUNSUPPORTED without the remap, PTYCHO_EINVAL
 * for z <= 0; on failure the previous geometry is kept. */
int ptycho_plan_set_distance(ptycho_plan_t* plan, double z);

/* Fractional scan offsets (f2 by the Fourier shift theorem, the paper's differentiable
 * scanning shift; Section "Benchmarking with state-of-art ...").  Registers delta, a DEVICE
 * array [L][J][2] of float32 (rows, then columns, in object pixels of wavelength l) that
 * every later compute call on this plan adds to the integer positions of the geometry: the
 * F x F window at pos[l][j] is resampled at r + delta[l][j] as F2^-1[ramp * F2 window],
 * ramp(k) = exp(2 pi i (f(k_y) d_y + f(k_x) d_x)), f in cycles per pixel with the Nyquist
 * index at -1/2; the window is taken as one period (its edge rows and columns wrap, where
 * the probe is negligible).  Any |delta| is accepted; large offsets belong in the integer
 * positions of a new plan.  The array stays owned by the caller and must stay alive while
 * registered; ptycho_step updates it in place when the Adam state has lr_delta > 0.
 * delta = NULL clears the registration (integer positions again).  The first registration
 * allocates the shift workspaces (3 x nsets x B x L x F^2 complex64).  PTYCHO_EUNSUPPORTED
 * when the plan processes a position's modes in chunks or T*M > 256 (T = 4, 8, 16, 16
 * threads per row for F = 64, 128, 256, 512); PTYCHO_ENOMEM when the workspaces do not fit;
 * the plain baseline (ptycho_plain_step) rejects plans with offsets. */
int ptycho_plan_set_offsets(ptycho_plan_t* plan, float* delta);

/* Object regularisation.  The paper adapts the loss with regularisers (Section "Universal
 * Ptychography Algorithm") and names L1 and total-variation regularisation of the object
 * amplitude (Section "3D structure information characterisation"); their exact forms are in its
 * Supplementary Information, which is not available, so this is a reading.  With the smoothed
 * amplitude a = sqrt(|O|^2 + eta^2) of every pixel of every object O_l,
 *   R = mu_l1 sum a + mu_tv sum sqrt(dx^2 + dy^2 + eta^2),
 *   dx = a[r][c+1] - a[r][c] (0 in the last column), dy = a[r+1][c] - a[r][c] (0 in the last row).
 * Adds R to *loss_dev (DEVICE double, may be NULL) and g = dR/dRe + i dR/dIm = (dR/da) O / a to
 * gO (packed objects, complex64, DEVICE), on stream.  mu_l1, mu_tv >= 0, eta > 0, all finite
 * (PTYCHO_EINVAL otherwise); mu_l1 = mu_tv = 0 launches nothing.  Deterministic (each pixel has
 * one owner; the value is summed in FP64 in a fixed order).  The first call allocates a small
 * per-tile partial buffer in the plan (PTYCHO_ENOMEM if that fails). */
int ptycho_regularise(ptycho_plan_t* plan, const float* O, float mu_l1, float mu_tv, float eta, float* gO,
                      double* loss_dev, void* stream);

/* One optimisation step on a batch of positions ("per batch" updates, Fig. 2 caption):
 * ptycho_adjoint into plan-owned gradient buffers (plus the object regulariser when the state
 * sets reg_l1 or reg_tv), then Adam on O (lr_O) and P (lr_P) in
 * place, and on sigma (lr_sigma > 0) and bg (lr_bg > 0) in place when the state asks for
 * it (sigma / bg must then be non-NULL; every component of sigma takes the Adam update,
 * with gradient 0 for positions outside the batch).  state->t is incremented on the host
 * before the update. */
int ptycho_step(ptycho_plan_t* plan, ptycho_adam_t* state, float* O, float* P, float* sigma,
                float* bg, const float* I_meas, const uint8_t* mask, int mask_per_frame,
                const int32_t* batch_idx, int nbatch, double* loss_dev, void* stream);

/* ptycho_step for a caller whose measured patterns and loss live in HOST memory (the paper
 * keeps its whole dataset resident on the GPU to avoid host-device transfers, Section
 * "Discussion"; this entry point is the form for data that stay on the host).  On stream:
 * I_meas_host (HOST, J*F*F floats, camera grid; page-locked memory makes the copy
 * asynchronous, pageable memory makes this call wait for it) is copied into the caller's
 * DEVICE buffer I_meas_dev (J*F*F floats; over all positions in order, batch by batch on a
 * plan-owned side stream that starts after the work already queued on stream, each position
 * batch's loss waiting only for its own frames, so the copies overlap the transforms of earlier
 * batches), ptycho_step runs on it with the other arguments
 * as documented there (loss_dev: DEVICE, 1 double, required here), and the loss is copied
 * into loss_host (HOST, 1 double), valid once the stream has passed this point.  The library
 * allocates nothing here.  PTYCHO_EINVAL for a NULL plan, I_meas_host, I_meas_dev, loss_dev
 * or loss_host, or a plan made on another device; PTYCHO_ECUDA when a copy cannot be
 * issued; otherwise the errors of ptycho_step. */
int ptycho_step_host(ptycho_plan_t* plan, ptycho_adam_t* state, float* O, float* P, float* sigma, float* bg,
                     const float* I_meas_host, float* I_meas_dev, const uint8_t* mask, int mask_per_frame,
                     const int32_t* batch_idx, int nbatch, double* loss_dev, double* loss_host, void* stream);

/* Number of kernel launches issued by the most recent compute call on this plan. */
int64_t ptycho_plan_last_launches(const ptycho_plan_t* plan);

/* Device-side status of the plan since the previous query, then cleared.  Bit 0
 * (PTYCHO_STATUS_BAD_INDEX): a batch_idx entry was outside [0, J); that position was
 * skipped.  Bit 1 (PTYCHO_STATUS_WAIT_TIMEOUT): a bulk shared-memory copy of a column pass
 * did not complete within about a second; the block gave up and its outputs for that call
 * are not valid.  Synchronises the device (call it outside the timed loop). */
#define PTYCHO_STATUS_BAD_INDEX 1
#define PTYCHO_STATUS_WAIT_TIMEOUT 2
int ptycho_plan_status(ptycho_plan_t* plan, int32_t* flags);

/* Plain (unfused) form of ptycho_step, the baseline the fused path is measured against:
 * every stage (gather, row DFT, column DFT, intensity, loss, R^T, multiply, inverse DFTs,
 * gradient scatter) is a separate kernel, exit waves go through a device buffer that the
 * call allocates (stream-ordered), and gradients are scattered with FP32 atomics (so their
 * summation order, and the last bits of the result, can vary between runs).  Arguments as
 * for ptycho_step with all positions; it updates O and P only (PTYCHO_EUNSUPPORTED when the
 * state asks for sigma or background updates). */
int ptycho_plain_step(ptycho_plan_t* plan, ptycho_adam_t* state, float* O, float* P, const float* sigma,
                      const float* bg, const float* I_meas, const uint8_t* mask, int mask_per_frame,
                      double* loss_dev, void* stream);

/* ---------------------------------------------------------------------------------------
 * Multi-site serving (continuous batching).  The paper reconstructs one dataset at a time;
 * this serves many reconstructions ("sites") of different F, J, L, M at once on one GPU.
 * Each admitted site keeps its plan, Adam moments (zero at admission), a device step
 * counter and its loss resident.  ptycho_server_tick runs one iteration of every active
 * site (forward, loss, adjoint, gradients, Adam over all its positions) as a single graph
 * launch, in one of two forms:
 *   PTYCHO_SERVE_SHARED_LAUNCHES: per frame size and per round of position batches,
 *     each pass of the pipeline is ONE kernel launch over the current batch of every active
 *     site of that frame size (a device work table assigns each block to a site); one launch
 *     each then reduces every site's loss, advances its step counter and runs its Adam.  The
 *     graph and tables are rebuilt when the active set changes (that rebuild synchronises the
 *     device).  These sites take the default pipeline variants and one scratch set: a geometry
 *     with flags or a zoom is rejected (PTYCHO_EUNSUPPORTED).  Each site's adjoint row pass runs
 *     in the variant its plan chose (per mode, or fused over the modes: one launch per block
 *     shape).
 *   PTYCHO_SERVE_SITE_GRAPHS (default): each site's own iteration graph (its plan's pipeline)
 *     is captured at admission and a tick launches one child-graph node per active site with
 *     no edges between them, so the sites' kernels overlap on the device.  Measured faster on
 *     the 64-request serving stream: 659 vs 517 K evaluations per second.
 * Sites are admitted between ticks while the HBM budget allows (their plan, moments and the
 * caller's resident O, P, I_meas and mask count against it) and give their memory back with
 * ptycho_server_release.  Results of a site do not depend on the other sites in the mix (no
 * shared buffers, per-site fixed-order reductions).  Host-driven: no kernel waits on another. */
#define PTYCHO_SERVE_SHARED_LAUNCHES 0
#define PTYCHO_SERVE_SITE_GRAPHS 1
typedef struct ptycho_server ptycho_server_t;

typedef struct {
  float* O; float* P;            /* DEVICE parameters, updated in place every iteration     */
  const float* I_meas;           /* DEVICE [J][F][F]                                        */
  const uint8_t* mask;           /* DEVICE mask or NULL, as for ptycho_loss                 */
  int32_t mask_per_frame;
  const float* sigma;            /* DEVICE [J] or NULL                                      */
  const float* bg;               /* DEVICE [F][F] or NULL                                   */
  float lr_O, lr_P, beta1, beta2, eps;   /* Adam hyper-parameters                           */
  int32_t iterations;            /* iterations to run before the site is done               */
} ptycho_site_t;

/* A server for the current device with a budget of device bytes and at most max_sites. */
int ptycho_server_create(int64_t hbm_budget_bytes, int32_t max_sites, ptycho_server_t** out);
/* Synchronises the device, frees every site and the server.  NULL is accepted. */
int ptycho_server_destroy(ptycho_server_t* server);
/* Validates and plans a site, checks the budget (PTYCHO_EBUSY when it does not fit or no
 * slot is free; nothing stays allocated then), allocates its state and captures its
 * iteration graph (per-site form).  *slot receives the site's slot.  Synchronous. */
int ptycho_server_admit(ptycho_server_t* server, const ptycho_geom_t* geom, const ptycho_site_t* site,
                        int32_t* slot);
/* Enqueues one iteration of every site that has iterations left, as one graph launch on
 * stream; *n_sites (may be NULL) receives how many sites it covered. */
int ptycho_server_tick(ptycho_server_t* server, void* stream, int32_t* n_sites);
/* Iterations enqueued so far and the loss of the last completed iteration (HOST double;
 * the copy synchronises with the device).  Either pointer may be NULL. */
int ptycho_server_site_status(ptycho_server_t* server, int32_t slot, int32_t* iters_done, double* loss);
/* Waits for the device, then frees the site's plan and state and returns its budget. */
int ptycho_server_release(ptycho_server_t* server, int32_t slot);
/* Bytes currently counted against the budget. */
int64_t ptycho_server_used_bytes(const ptycho_server_t* server);
/* Selects the form of the tick (PTYCHO_SERVE_SHARED_LAUNCHES or PTYCHO_SERVE_SITE_GRAPHS);
 * only while no site is admitted (PTYCHO_EINVAL otherwise, or for another mode). */
int ptycho_server_set_mode(ptycho_server_t* server, int32_t mode);

/* Opt-in per-kernel timing.  While enabled, every launch of a compute call is bracketed
 * by a CUDA event pair recorded on the call's stream.  ptycho_plan_profile_read waits for
 * the recorded events and fills, per kernel kind (PTYCHO_K_*), the summed device time in
 * ms and the launch count since profiling was enabled or last read; then it restarts.
 * ms and launches are HOST arrays of PTYCHO_NUM_KERNELS entries. */
#define PTYCHO_K_ROW_FWD 0       /* exit wave + row DFT                                  */
#define PTYCHO_K_COL_FWD 1       /* column DFT + |Psi|^2 mode sum                         */
#define PTYCHO_K_LOSS 2          /* remap + mask + loss partials + dL/dI                  */
#define PTYCHO_K_COL_ADJ 3       /* R^T, (2/F) G Psi, inverse column DFT                  */
#define PTYCHO_K_ROW_ADJ 4       /* inverse row DFT + probe gradient                      */
#define PTYCHO_K_OBJ_GRAD 5      /* tile-owned object-gradient sum                        */
#define PTYCHO_K_LOSS_REDUCE 6   /* FP64 loss reduction                                   */
#define PTYCHO_K_ADAM 7          /* Adam update                                          */
#define PTYCHO_K_REMAP_ADJ 8     /* R^T of the tilted-plane remap                         */
#define PTYCHO_K_SHIFT 9         /* Fourier shift of fractional scan offsets + dL/ddelta  */
#define PTYCHO_K_REG 10          /* object regulariser (value and gradient)               */
#define PTYCHO_K_RES_FWD 11      /* frame-resident forward: exit waves, 2D DFT, |Psi|^2 sum */
#define PTYCHO_K_RES_ADJ 12      /* frame-resident adjoint: Psi recomputed, chi, gradients  */
#define PTYCHO_NUM_KERNELS 13
int ptycho_plan_profile(ptycho_plan_t* plan, int enable);
int ptycho_plan_profile_read(ptycho_plan_t* plan, double* ms, int64_t* launches);
const char* ptycho_kernel_name(int kind);

/* Allocation-free forward model.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc while they run (an application that gives all
 * device memory to its own pool at start-up, a latency-critical loop that cannot take the
 * synchronisation an allocation may cause, a deployment that bans allocation after
 * initialisation).  It computes exactly what ptycho_forward computes for a plan without
 * the tilted-plane remap, but needs no plan: every intermediate lives in one fixed device
 * array of PTYCHO_NOALLOC_SCRATCH_BYTES (32 MiB) that each GPU loading this library holds
 * until the process exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *   L, M, F, J, obj_h, obj_w  as in ptycho_geom_t (HOST arrays)
 *   pos     HOST [L][J][2] scan positions, validated like ptycho_plan_create (PTYCHO_ERANGE)
 *   O, P, sigma, bg, I_pred  DEVICE arrays as in ptycho_forward
 * Returns PTYCHO_ETOOLARGE when the position tables plus one complex and one real frame
 * exceed the fixed array; larger mode counts are processed in chunks that fit.
 * Set-up: the first call on each device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  The small host tables
 * are copied with cudaMemcpyAsync from pageable memory, so the call waits for the stream's
 * earlier work before it returns.  All calls share the one array and it keeps the previous
 * call's contents: calls whose work overlaps on the GPU (other streams, other threads)
 * race and must be serialised by the caller. */
#define PTYCHO_NOALLOC_SCRATCH_BYTES (32u << 20)
int ptycho_forward_noalloc(int32_t L, int32_t M, int32_t F, int32_t J, const int32_t* obj_h,
                           const int32_t* obj_w, const int32_t* pos, const float* O, const float* P,
                           const float* sigma, const float* bg, float* I_pred, void* stream);

/* Data-side tilt correction: the tilted-plane remap of the measurement model (f5 of Eq. 2)
 * applied once to the measured patterns instead of inside the model, the way the paper
 * preprocesses its reflection data (Section "Experimental setup and ptychography
 * reconstruction": each pattern is interpolated non-uniformly onto a grid uniform in
 * sample-plane spatial frequency, the correction yields the mask of the reduced field of
 * view, and pixels outside the value thresholds are discarded).  The corrected patterns are
 * fitted by a plan built with remap = 0, passing the mask with mask_per_frame = 1.
 * The model grid is that of the in-model remap: F x F, zero frequency at (F/2, F/2),
 * spacings db = (p/z) cos(tilt) along rows and da = p/z along columns in the reflected
 * ray's in-plane direction cosines.  Model pixel (i, k) has b = (i - F/2) db and
 * a = (k - F/2) da; rotated by the tilt about the camera x axis its ray is (a, b + sin, w),
 * w = sqrt(1 - a^2 - (b + sin)^2) >= 0 (it leaves the sample surface), so in the camera frame
 * d_y = (b + sin) cos - w sin and d_z = (b + sin) sin + w cos, and it meets the camera at
 * X = z a / d_z, Y = z d_y / d_z: fractional camera index (Y/p + F/2, X/p + F/2), evaluated in
 * FP64 with every operation rounded separately.  The output is the bilinear interpolation of
 * the camera pattern there.  A model pixel is kept (mask 1) when the ray exists (w^2 > 0,
 * d_z > 0), its four camera taps lie inside the crop (0 <= y < F-1, 0 <= x < F-1) and every
 * tap value v satisfies lo <= v < hi (the paper's thresholds are 4 and 65535; pass -INFINITY
 * and INFINITY for the field-of-view mask alone).
 *   F          side of the camera crop and of the model grid, 2..8192
 *   J          number of patterns; 0 launches nothing
 *   z, det_pixel, tilt_rad   distance to the camera (m), camera pixel pitch (m) and tilt from
 *              the sample normal (|tilt| < pi/2), as in ptycho_geom_t
 *   I_cam      DEVICE [J][F][F] float, camera-grid patterns, zero frequency at (F/2, F/2)
 *   I_model    DEVICE [J][F][F] float, out: corrected patterns, 0 where the mask is 0; must
 *              not overlap I_cam
 *   mask       DEVICE [J][F][F] uint8, out, or NULL: 1 = kept, 0 = not kept
 * Asynchronous on stream.  The camera positions are computed first (ptycho_tilt_table) into a
 * table that this call allocates stream-ordered (cudaMallocAsync) and frees again; callers that
 * correct many stacks with one geometry build the table once and call ptycho_tilt_apply.
 * PTYCHO_EINVAL for a bad size, geometry or threshold pair (NaN or lo >= hi), a NULL array with
 * J > 0, or overlapping inputs and outputs; PTYCHO_ENOMEM when the table cannot be allocated. */
int ptycho_tilt_correct(int32_t F, int64_t J, double z, double det_pixel, double tilt_rad, const float* I_cam,
                        float lo, float hi, float* I_model, uint8_t* mask, void* stream);

/* Bytes of the tilt-correction table of an F x F grid (20 per model pixel: four FP32 bilinear
 * weights, then one int32 camera offset of the top-left tap, -1 for a pixel that is never
 * kept), or -1 when F is outside 2..8192. */
int64_t ptycho_tilt_table_bytes(int32_t F);

/* Fills a caller-owned DEVICE table (ptycho_tilt_table_bytes(F) bytes, 16-byte aligned) with
 * the camera position of every model pixel for this geometry, as ptycho_tilt_correct defines
 * it.  Asynchronous on stream; PTYCHO_EINVAL for a bad size or geometry, a NULL or misaligned
 * table. */
int ptycho_tilt_table(int32_t F, double z, double det_pixel, double tilt_rad, void* table, void* stream);

/* The interpolation and masking of ptycho_tilt_correct with a table from ptycho_tilt_table
 * (same F); the result is identical to ptycho_tilt_correct's for that geometry.  Arguments and
 * errors as for ptycho_tilt_correct; the outputs must not overlap the table. */
int ptycho_tilt_apply(int32_t F, int64_t J, const void* table, const float* I_cam, float lo, float hi,
                      float* I_model, uint8_t* mask, void* stream);

/* Static text for a return code. */
const char* ptycho_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* PTYCHO_GB300_H */
