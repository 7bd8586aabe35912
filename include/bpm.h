/*
 * bpm.h - C ABI of the B300 split-step beam-propagation library (libbpm.so).
 *
 * The library propagates a complex scalar field slice by slice through a
 * refractive-index volume with the beam-propagation method and the exact
 * propagator, as in Biobeam (Weigert, Myers & Kreysing, arXiv:1706.02261,
 * method paragraph), and synthesises the multiplexed focused input fields the
 * paper introduces in the same paragraph.  For every slice z:
 *
 *     E <- IDFT2( H . DFT2(E) ),  H = exp(i kz dz) where kz^2 > 0, else 0,
 *          kz = sqrt((k0 n0)^2 - kx^2 - ky^2), k0 = 2 pi / lambda
 *     E <- E . exp(i k0 dn(x, y, z) dz),        dn = n - n0
 *     I[z] = |E|^2                              (the excitation at every voxel,
 *                                                light-sheet paragraph)
 *
 * Conventions for every call:
 *  - Pointers named d_* are DEVICE pointers owned by the caller; h_* are host
 *    pointers.  Device arrays must be 16-byte aligned (BPM_ERR_ALIGN otherwise).
 *  - Fields are interleaved complex float (re, im), row-major [ny][nx]
 *    (x fastest).  Index volumes are IEEE half dn = n - n0, z-major
 *    [nz][ny][nx].  Intensity volumes are float, [nz][ny][nx].
 *  - Lengths are micrometres; lambda is the vacuum wavelength; kx follows the
 *    DFT bin order 0, 1, ..., then the negative bins; periodic boundaries.
 *  - Work is enqueued asynchronously on the given stream (0 = legacy default
 *    stream).  Argument errors are returned immediately; errors found on the
 *    device (barrier timeout, non-finite index values) are returned by
 *    bpm_check(), which synchronises the stream of the plan's last call.
 *  - Every function returns BPM_OK (0) or a negative BPM_ERR_* code and never
 *    aborts; bpm_last_error() gives a message for the calling thread.
 *  - A plan may be used from one host thread / one stream at a time.
 */
#ifndef BPM_H
#define BPM_H

#include <stddef.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    BPM_OK = 0,
    BPM_ERR_ARG = -1,          /* invalid argument (size, range, NULL)          */
    BPM_ERR_ALIGN = -2,        /* a device pointer is not 16-byte aligned       */
    BPM_ERR_CUDA = -3,         /* a CUDA runtime call failed                    */
    BPM_ERR_TIMEOUT = -4,      /* a device-side barrier wait ran out of time    */
    BPM_ERR_NAN = -5,          /* non-finite value in the refractive-index data */
    BPM_ERR_UNSUPPORTED = -6   /* grid size or configuration not supported      */
};

/* Plan flags. */
#define BPM_FLAG_SYNC          0x1u  /* every call synchronises and reports device errors */
#define BPM_FLAG_MULTI_LAUNCH  0x2u  /* one kernel launch per half-step instead of the
                                        persistent kernel (comparison path)           */
#define BPM_FLAG_GRAPH         0x4u  /* batched plans: capture the launch in a CUDA graph
                                        once per argument set and replay it          */
#define BPM_FLAG_ADAPTIVE      0x8u  /* single-instance plans: locally adapted expansion
                                        of the index (method paragraph), reading B:
                                        slice z takes its mean index step delta_z as
                                        reference, propagator H exp(i delta_z k0^2 n0
                                        dz / kz0) (exact medium n0 + delta_z to first
                                        order), screen exp(i k0 (dn - delta_z) dz); the
                                        means are computed on the device per call
                                        (one extra read of the index slices)          */

typedef struct bpm_plan_s *bpm_plan_t;

/* One propagation problem (one field): rows of nx points along x, ny rows
 * along y, nz slices.  nx and ny must each be one of 64, 96, 128, 192, 256,
 * 384, 512, 768, 1024, 1536, 2048 (the products of 2 and 3 the FFT kernels are
 * built for) with nx * ny <= 2^22, e.g. the 1024 x 2048 lateral grid of the
 * paper's 10^6-PSF calculation (light-sheet paragraph); nz >= 0.  Batched
 * plans (several instances) take square grids of 64, 128, 192, 256, 384, 512
 * or 1024.  dx, dy, dz, lambda and n0 must be positive.  tilt_x, tilt_y are
 * unused by the propagation and reserved for input helpers. */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, lambda, n0;
    double tilt_x, tilt_y;
} bpm_instance_desc;

/* bpm_plan - validate n_inst problem descriptions and build everything the
 * propagation needs that does not depend on the field: the propagator table
 * H = exp(i (kz - k0 n0) dz) / (nx ny) per instance (the carrier exp(i k0 n0 dz)
 * is factored out and applied in FP64 at the end; the 1/(nx ny) of the inverse
 * DFT is folded in), computed in FP64 on the device and stored as complex
 * float; the FFT twiddle tables; the team/launch configuration; barrier and
 * error words.  The plan owns this device memory (about 8 bytes per lateral
 * pixel per instance plus a few KiB).  The method paragraph of the paper
 * defines the exact propagator; the evanescent cut maps kz^2 <= 0 to 0.
 *   out     : receives the plan handle (set to NULL on failure)
 *   inst    : host array of n_inst descriptions (1 <= n_inst <= 4096)
 *   flags   : BPM_FLAG_* bits
 *   stream  : stream on which the table kernels run
 * Errors: BPM_ERR_ARG, BPM_ERR_UNSUPPORTED, BPM_ERR_CUDA. */
int bpm_plan(bpm_plan_t *out, const bpm_instance_desc *inst, int n_inst, unsigned flags,
             cudaStream_t stream);

/* bpm_propagate - run slices [z_begin, z_end) of every instance (clamped to
 * [0, nz_i)), i.e. the split-step loop of the method paragraph: per slice the
 * forward 2D DFT, the propagator multiply, the inverse 2D DFT, the phase screen
 * exp(i k0 dn dz) and the intensity |E|^2.  A single-instance plan runs the
 * whole loop in one cooperative persistent launch in which all SMs share the
 * field, for square grids and grids whose sides differ by a factor of two;
 * other grids (and BPM_FLAG_MULTI_LAUNCH) take one launch per half-step
 * (bpm_plan_info reports which).  A plan with several instances (any
 * mix of the supported sizes) runs all of them in one persistent launch of
 * thread-block clusters: each cluster propagates whole instances taken from a
 * device work queue, largest first, while a second launch of two-CTA teams
 * on the SMs the clusters leave free takes small instances from the other
 * end of the queue (with BPM_FLAG_GRAPH both launches and the argument upload
 * are one CUDA graph, captured once per argument set).
 *   d_dn   : host array of n_inst device pointers; instance i reads the FP16
 *            volume [nz_i][ny][nx] (slice z at offset z*nx*ny)
 *   d_Ein  : host array of device pointers to the input fields (entrance of
 *            slice z_begin)
 *   d_Eout : host array of device pointers receiving the field after slice
 *            z_end-1, including the carrier exp(i k0 n0 dz (z_end - z_begin));
 *            d_Eout[i] may equal d_Ein[i] (in-place); d_Eout[i] is also the
 *            working buffer during the call
 *   d_I    : NULL, or a host array of device pointers (entries may be NULL)
 *            to [nz_i][ny][nx] float volumes; slice z receives |E|^2 after
 *            slice z's screen (only slices in [z_begin, z_end) are written)
 * Errors: BPM_ERR_ARG, BPM_ERR_ALIGN, BPM_ERR_CUDA; device errors via bpm_check. */
int bpm_propagate(bpm_plan_t p, const void *const *d_dn, const void *const *d_Ein,
                  void *const *d_Eout, float *const *d_I, int z_begin, int z_end,
                  cudaStream_t stream);

/* bpm_propagate_window - bpm_propagate with an intensity window per
 * instance: instance i computes |E|^2 only for slices z in
 * [h_w_begin[i], h_w_end[i]) (and in [z_begin, z_end)), into d_I[i] laid out
 * [h_w_end[i] - h_w_begin[i]][ny][nx] with slice z at offset
 * (z - h_w_begin[i])*nx*ny.  This is how a PSF sweep writes only the slices
 * around the foci (the paper's multiplexing scheme: each multiplexed field is
 * needed near its focal depth only, and propagation can stop at the window's
 * end by z_end).  bpm_propagate is this call with windows [0, nz_i).
 *   h_w_begin, h_w_end : host arrays of n_inst ints, 0 <= w_begin <= w_end
 * Other arguments and errors as bpm_propagate. */
int bpm_propagate_window(bpm_plan_t p, const void *const *d_dn, const void *const *d_Ein,
                         void *const *d_Eout, float *const *d_I, int z_begin, int z_end,
                         const int *h_w_begin, const int *h_w_end, cudaStream_t stream);

/* bpm_propagate_reverse - the split-step loop towards -z through slices
 * z_end-1, z_end-2, ..., z_begin of a single-instance plan (the same
 * per-slice step: propagator over dz, then the slice's screen), e.g. light
 * emitted inside the sample travelling back to its surface: the field enters
 * at the exit plane of slice z_end-1 and d_Eout receives it at the entrance
 * plane of slice z_begin (with the carrier exp(i k0 n0 dz (z_end - z_begin))).
 * d_I (nullable) is the [nz][ny][nx] volume; slice z receives |E|^2 after its
 * screen.  With BPM_FLAG_ADAPTIVE each slice uses its own mean index step.
 * The paper's adaptive-optics simulation (conjugating the wavefront of a
 * guide star at the sample surface, Fig. 2c paragraph) is this call,
 * bpm_phase_conjugate, and a forward bpm_propagate.
 * Errors: as bpm_propagate; BPM_ERR_UNSUPPORTED for batched plans. */
int bpm_propagate_reverse(bpm_plan_t p, const void *d_dn, const void *d_Ein, void *d_Eout, float *d_I,
                          int z_begin, int z_end, cudaStream_t stream);

/* bpm_propagate_absorbing - bpm_propagate of a single-instance plan with a
 * complex refractive index n = n0 + dn + i kappa (the paper's phantoms may
 * absorb: adaptive-optics paragraph): each slice's screen is
 * exp(i k0 (dn + i kappa) dz) = exp(i k0 dn dz) exp(-k0 kappa dz).
 *   d_kappa : device FP16 volume [nz][ny][nx] of kappa (>= 0 absorbs), 16-byte
 *             aligned; each value read once (global streaming loads)
 * Other arguments as bpm_propagate.  Errors: as bpm_propagate;
 * BPM_ERR_UNSUPPORTED for batched plans and with BPM_FLAG_ADAPTIVE. */
int bpm_propagate_absorbing(bpm_plan_t p, const void *d_dn, const void *d_kappa, const void *d_Ein,
                            void *d_Eout, float *d_I, int z_begin, int z_end, cudaStream_t stream);

/* bpm_phase_conjugate - E <- conj(E) in place on instance inst's field (the
 * time-reversed monochromatic wave).  d_E: device complex float [ny][nx],
 * 16-byte aligned.  Errors: BPM_ERR_ARG, BPM_ERR_ALIGN, BPM_ERR_CUDA. */
int bpm_phase_conjugate(bpm_plan_t p, int inst, void *d_E, cudaStream_t stream);

/* bpm_demultiplex - cut one patch per focus out of an intensity window, the
 * de-multiplexing step of the paper's multiplexed PSF calculation (a set of
 * non-overlapping PSFs computed in one propagation is split into the
 * individual PSFs).  Patch j is
 *   d_out[j][k][y][x] = I(iz_j - pz/2 + k, iy_j - py/2 + y, ix_j - px/2 + x)
 * for k < pz, y < py, x < px, with lateral indices taken modulo the grid size
 * (the periodic boundary of the propagation) and 0 for slices outside the
 * window [w_begin, w_begin + w_nz).
 *   inst     : instance whose grid (nx, ny) is used
 *   d_I      : device float window [w_nz][ny][nx] (slice z at (z - w_begin)*nx*ny)
 *   h_foci   : host array of n_foci (ix, iy, iz) voxel triples, 0 <= ix < nx, 0 <= iy < ny
 *   d_out    : device float [n_foci][pz][py][px], written with streaming stores
 * Errors: BPM_ERR_ARG (focus outside the grid, bad sizes, NULL), BPM_ERR_CUDA. */
int bpm_demultiplex(bpm_plan_t p, int inst, const float *d_I, int w_begin, int w_nz, int n_foci,
                    const int *h_foci, int px, int py, int pz, float *d_out, cudaStream_t stream);

/* bpm_propagate_static - the same propagation as bpm_propagate for one
 * instance, for callers that cannot allocate device memory.  Some callers run
 * inside a host application whose allocator owns the whole device (cudaMalloc
 * would fail or break its accounting), or in a loop where the device-wide
 * synchronisation of cudaMalloc/cudaFree is not acceptable, or must not risk
 * an out-of-memory failure after start-up.  This entry point allocates nothing
 * and needs no plan: the propagator table, the twiddle tables, the barrier
 * counter and the error word live in one fixed array of device memory inside
 * the library (about 528 KiB), which every GPU that loads the library keeps
 * until the process exits.  The paper has no counterpart; it is a service of
 * this library.
 *   inst          : one problem description; nx = ny must be 64, 96, 128,
 *                   192 or 256 (larger or rectangular grids return
 *                   BPM_ERR_UNSUPPORTED: the fixed array holds the propagator
 *                   of a 256 x 256 grid at most)
 *   d_dn, d_Ein, d_Eout, d_I, z_begin, z_end : as for bpm_propagate, for this
 *                   one instance (d_I may be NULL)
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the rest of
 * the process; make that first call before any stream capture.  The kept
 * address belongs to the device's current context: after cudaDeviceReset on
 * that device it is stale, so do not call this function again on a device
 * that has been reset.  Every call rebuilds the tables and clears the counter
 * and error word on `stream`, runs the propagation, then synchronises `stream`
 * and returns the device status (BPM_ERR_TIMEOUT, BPM_ERR_NAN) directly.  All
 * calls on a device share the array, so calls that overlap on the GPU (other
 * streams, other host threads) race and give wrong results; issue them one at
 * a time.
 * Errors: BPM_ERR_ARG, BPM_ERR_ALIGN, BPM_ERR_UNSUPPORTED, BPM_ERR_CUDA,
 * BPM_ERR_TIMEOUT, BPM_ERR_NAN. */
int bpm_propagate_static(const bpm_instance_desc *inst, const void *d_dn, const void *d_Ein,
                         void *d_Eout, float *d_I, int z_begin, int z_end, cudaStream_t stream);

/* bpm_propagate_host - bpm_propagate of all nz slices of a single-instance
 * plan with HOST index and intensity volumes: the library streams the FP16
 * index volume to the device and the intensity volume back in chunks of
 * `chunk` slices through two device ring slots, so that the host->device
 * copies, the propagation (one persistent launch per chunk, the field staying
 * on the device) and the device->host copies overlap on three streams.
 *   h_dn   : host [nz][ny][nx] FP16 index volume
 *   Ein    : input field, host memory (ein_on_device = 0) or device memory
 *            (ein_on_device = 1, e.g. from bpm_multiplex_psf)
 *   h_Eout : host [ny][nx] complex float, receives the field after the volume
 *   h_I    : NULL or host [nz][ny][nx] float, receives |E|^2 per slice
 * Host buffers should be page-locked (cudaHostAlloc/cudaHostRegister; torch's
 * pin_memory) for the copies to overlap; pageable buffers work but serialise.
 * The plan owns the ring (2 * chunk * nx * ny * 6 bytes, allocated on the
 * first call or when a larger chunk is requested).  Synchronous: returns when
 * h_Eout and h_I are complete, with the device status (as bpm_check).
 * Errors: BPM_ERR_ARG, BPM_ERR_ALIGN, BPM_ERR_UNSUPPORTED (batched plans),
 * BPM_ERR_CUDA, BPM_ERR_TIMEOUT, BPM_ERR_NAN. */
int bpm_propagate_host(bpm_plan_t p, const void *h_dn, const void *Ein, int ein_on_device, void *h_Eout,
                       float *h_I, int chunk, cudaStream_t stream);

/* bpm_multiplex_psf - the multiplexed input field of the method paragraph:
 * the sum of n_foci focused fields, one per emitter.  Emitter j sits at the
 * grid point nearest to (h_xyz[3j], h_xyz[3j+1]) (rounded in FP64 as
 * floor(x/dx + 0.5)) with phase h_phase[j], and focuses at depth h_xyz[3j+2]
 * after forward propagation: its spectrum is cut to the scalar pupil
 * |k_perp| <= k0 NA (propagating waves only) and multiplied by
 * exp(-i kz z_j).  Each emitter has amplitude sqrt(nx ny / n_pupil), so each
 * focused field has unit energy sum |E|^2 = 1 before the summation.  Emitters
 * sharing a depth are synthesised together (one FFT pair per distinct depth).
 * Emitters outside the grid are skipped.
 *   inst   : instance index whose grid is used
 *   n_foci : 0 <= n_foci <= 1048576
 *   d_Eout : device [ny][nx] complex float, overwritten
 * Errors: BPM_ERR_ARG, BPM_ERR_ALIGN, BPM_ERR_CUDA. */
int bpm_multiplex_psf(bpm_plan_t p, int inst, int n_foci, const double *h_xyz,
                      const double *h_phase, double NA, void *d_Eout, cudaStream_t stream);

/* bpm_multiplex_annular - bpm_multiplex_psf with the annular pupil
 * NA_in <= |k_perp| / k0 <= NA_out: each emitter becomes a Bessel beam
 * (propagation-invariant as the annulus narrows), and a row of emitters a
 * Bessel lattice, one of the paper's illumination modalities (light-sheet
 * modalities paragraph).  Unit energy per emitter; the pupil membership is
 * decided in FP64 as for the disk.  NA_in = 0 is bpm_multiplex_psf.
 * Errors: as bpm_multiplex_psf; BPM_ERR_ARG unless 0 <= NA_in < NA_out. */
int bpm_multiplex_annular(bpm_plan_t p, int inst, int n_foci, const double *h_xyz, const double *h_phase,
                          double NA_in, double NA_out, void *d_Eout, cudaStream_t stream);

/* bpm_light_sheet - cylindrical light sheet (the paper's Fig. 2a illumination,
 * NA 0.15): thin along x, uniform along y; angular spectrum
 * exp(-(kx w0 / 2)^2) on the ky = 0 line, w0 = lambda / (pi NA), centred at
 * x_c = (nx/2) dx, defocused by exp(-i kz zf) (propagating waves only) and
 * scaled so that |E|^2 = 1 at (x_c, zf) after exact propagation.
 *   d_Eout : device [ny][nx] complex float, overwritten
 * Errors: BPM_ERR_ARG, BPM_ERR_ALIGN, BPM_ERR_CUDA. */
int bpm_light_sheet(bpm_plan_t p, int inst, double NA, double zf, void *d_Eout,
                    cudaStream_t stream);

/* bpm_check - wait for the plan's last stream and return the first device
 * error recorded since the previous bpm_check (BPM_ERR_TIMEOUT, BPM_ERR_NAN),
 * clearing it; BPM_OK otherwise. */
int bpm_check(bpm_plan_t p);

/* bpm_free - release the plan's device memory (synchronises its stream).
 * NULL is accepted.  The handle must not be used afterwards. */
int bpm_free(bpm_plan_t p);

/* bpm_last_error - message for the last failing call on this host thread. */
const char *bpm_last_error(void);

/* bpm_plan_info - launch configuration chosen for the plan, for reports:
 * out[0] = team CTAs, out[1] = threads per CTA, out[2] = dynamic shared
 * memory bytes, out[3] = persistent (1) or multi-launch (0), out[4] = kernel
 * launches per bpm_propagate call, out[5] = transform schedule in use,
 * out[6] = number of schedules of the plan's grid size (batched plans: the
 * schedule set of the batched kernel and the number of sets).  n_out may be
 * smaller than 7. */
int bpm_plan_info(bpm_plan_t p, int *out, int n_out);

/* bpm_autotune - time the propagation of slices [0, z_probe) on the given
 * buffers and keep the fastest configuration for later calls (this is where
 * the team sizes and radix schedules of batched propagation are picked).  Batched
 * plans: every instance, with each transform schedule set of the batched
 * kernel (three sets of radix order and pass structure for the 256, 512 and
 * 1024 transforms) and each cluster size (2, 4, 8, 16 CTAs per team).
 * Single-field plans: each transform schedule of the grid size (radix order
 * and pass structure of the row and column transforms: square grids of 256
 * and 512 have three, 1024 two, the other grids one).  Overwrites d_Eout and
 * the first z_probe intensity slices; synchronises the stream (and the device
 * when the schedule changes).  Errors: BPM_ERR_ARG, BPM_ERR_CUDA. */
int bpm_autotune(bpm_plan_t p, const void *const *d_dn, const void *const *d_Ein, void *const *d_Eout,
                 float *const *d_I, int z_probe, cudaStream_t stream);

/* bpm_set_schedule - use transform schedule `schedule` (0 .. out[6] - 1 of
 * bpm_plan_info).  Single-field plans: a square plan starts with the schedule
 * measured fastest for its size, 2 for 512 and 0 for the others; the rows and
 * columns of a rectangular grid each take their length's.  Batched plans: the
 * schedule set of the batched kernel (starts at 0).  Results of every
 * schedule agree to FP32 rounding.  Synchronises the device when the schedule
 * changes.  Errors: BPM_ERR_ARG (NULL plan, schedule out of range), BPM_ERR_CUDA. */
int bpm_set_schedule(bpm_plan_t p, int schedule);

/* bpm_debug_set_barrier_timeout - test hook: device barrier wait limit in
 * nanoseconds for this plan (default 2e9), and an extra count added to the
 * barrier target so that a barrier can be made to run out on purpose (0 in
 * normal use).  A barrier that runs out records BPM_ERR_TIMEOUT and every CTA
 * leaves the kernel. */
int bpm_debug_set_barrier_timeout(bpm_plan_t p, unsigned long long timeout_ns,
                                  unsigned extra_arrivals);

/* bpm_debug_stall_exchange - test hook for the bounded wait of the field
 * exchange between the half-steps of a single-field persistent launch (each
 * element carries the parity of the half-step that wrote it; consumers poll
 * their elements).  With on != 0 the entrance field's forward transform
 * writes the parity the row half-steps write later, so the first column
 * half-step waits for a value that never comes: the wait runs out after the
 * plan's limit (bpm_debug_set_barrier_timeout), records BPM_ERR_TIMEOUT and
 * every CTA leaves the kernel, leaving the context usable.  Batched plans:
 * the same for their instances that use the exchange (sides up to 192); the
 * setting is read when the batched launch is made, so plans with
 * BPM_FLAG_GRAPH keep the value their graph was captured with.  0 in normal
 * use; plans that run one launch per half-step ignore it.  Errors:
 * BPM_ERR_ARG. */
int bpm_debug_stall_exchange(bpm_plan_t p, int on);

#ifdef __cplusplus
}
#endif
#endif /* BPM_H */
