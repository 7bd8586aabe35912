/*
 * FP64 CPU oracle for split-step beam propagation with the exact propagator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference against
 * which the CUDA path is checked.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant with the CUDA library and must never be linked into it.
 *
 * What it computes (Weigert, Myers & Kreysing, "Biobeam", arXiv:1706.02261,
 * method paragraph: a beam-propagation model with the exact propagator, a
 * refractive-index screen per slice, and multiplexed focused input fields; the
 * light-sheet paragraph: the excitation is the intensity at every voxel):
 *
 *   k0 = 2 pi / lambda,  K = k0 n0,  kx = 2 pi fftfreq(nx, dx), ky likewise
 *   H(kx,ky) = exp(i sqrt(K^2 - kx^2 - ky^2) dz)  if K^2 - kx^2 - ky^2 > 0
 *            = 0                                  otherwise (evanescent cut)
 *   for each slice z:
 *       E <- IDFT2( H * DFT2(E) )          (DFT2 unnormalised, IDFT2 has 1/(nx ny))
 *       E <- E * exp(i k0 dn[z] dz)        (phase screen, dn = n - n0)
 *       I[z] = |E|^2
 *
 * Locally adapted expansion, reading B (oracle_bpm_adaptive).  The method
 * paragraph pairs the exact propagator with "a locally adapted expansion of
 * refractive indices" (its supplementary notes are not available).  Reading B
 * takes, per slice, the slice's mean index n0 + delta_z as the reference:
 *   delta_z = (1 / (nx ny)) sum over the slice of dn[z]
 *   H_z(kx,ky) = exp(i (kz0 + delta_z k0^2 n0 / kz0) dz)  if kz0^2 > 0, else 0,
 *            kz0 = sqrt(K^2 - kx^2 - ky^2)
 *     (the exact propagator of the medium n0 + delta_z to first order in
 *      delta_z: d kz / d n = k0^2 n / kz)
 *   E <- IDFT2( H_z * DFT2(E) ),  E <- E * exp(i k0 (dn[z] - delta_z) dz)
 * so a slice of uniform index is propagated by the propagator of its own
 * medium (to first order) instead of the background's propagator and a screen.
 *
 * Every step follows that definition literally: no carrier factoring, no fused
 * passes, no reordering.  The DFT is a recursive mixed-radix decimation in time
 * (smallest prime factor first, a direct O(n^2) sum for prime lengths), with
 * twiddles evaluated by cos/sin of the reduced exponent in double precision.
 *
 * Layout: complex arrays are interleaved (re, im) doubles, row-major [y][x];
 * the dn volume is [z][y][x] doubles (the FP16 values of the CUDA path widened
 * exactly).  All sizes are in elements, lengths in micrometres.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double kTwoPi = 6.283185307179586476925286766559;

/* exp(sign * 2 pi i * m / n), with m reduced modulo n first so the argument
 * stays in [0, 2 pi). */
static cplx root_of_unity(long long m, long long n, int sign)
{
    long long r = m % n;
    if (r < 0) r += n;
    double a = kTwoPi * (double)r / (double)n;
    return cos(a) + (double)sign * sin(a) * I;
}

static int smallest_factor(int n)
{
    for (int p = 2; (long long)p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* out[k] = sum_j in[j*stride] exp(sign 2 pi i j k / n), k in [0, n).
 * Decimation in time: with n = p m (p the smallest prime factor), the p
 * interleaved sub-sequences in[a + p j] are transformed recursively, then each
 * output k' + b m gathers sum_a W_n^{a (k' + b m)} Y_a[k']. */
static void dft_rec(int n, const cplx *in, int stride, cplx *out, int sign)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int p = smallest_factor(n);
    if (p == n) {
        for (int k = 0; k < n; ++k) {
            cplx acc = 0;
            for (int j = 0; j < n; ++j)
                acc += in[(long long)j * stride] * root_of_unity((long long)j * k, n, sign);
            out[k] = acc;
        }
        return;
    }
    int m = n / p;
    for (int a = 0; a < p; ++a)
        dft_rec(m, in + (long long)a * stride, stride * p, out + (long long)a * m, sign);
    cplx tbuf[64], ubuf[64];
    cplx *t = p <= 64 ? tbuf : (cplx *)malloc(sizeof(cplx) * (size_t)p);
    cplx *u = p <= 64 ? ubuf : (cplx *)malloc(sizeof(cplx) * (size_t)p);
    for (int k = 0; k < m; ++k) {
        for (int a = 0; a < p; ++a)
            t[a] = out[(long long)a * m + k];
        for (int b = 0; b < p; ++b) {
            cplx acc = 0;
            for (int a = 0; a < p; ++a)
                acc += t[a] * root_of_unity((long long)a * (k + (long long)b * m), n, sign);
            u[b] = acc;
        }
        for (int b = 0; b < p; ++b)
            out[k + (long long)b * m] = u[b];
    }
    if (p > 64) {
        free(t);
        free(u);
    }
}

/* In-place unnormalised 1D DFT of length n; sign = -1 forward, +1 inverse. */
int oracle_dft1(int n, double *x, int sign)
{
    if (n < 1 || (sign != 1 && sign != -1)) return -1;
    cplx *buf = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *src = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    memcpy(src, x, sizeof(cplx) * (size_t)n);
    dft_rec(n, src, 1, buf, sign);
    memcpy(x, buf, sizeof(cplx) * (size_t)n);
    free(buf);
    free(src);
    return 0;
}

/* In-place unnormalised 2D DFT of a row-major [ny][nx] array: every row, then
 * every column. */
int oracle_dft2(int nx, int ny, double *xv, int sign)
{
    if (nx < 1 || ny < 1 || (sign != 1 && sign != -1)) return -1;
    cplx *x = (cplx *)xv;
#pragma omp parallel
    {
        int nmax = nx > ny ? nx : ny;
        cplx *src = (cplx *)malloc(sizeof(cplx) * (size_t)nmax);
        cplx *dst = (cplx *)malloc(sizeof(cplx) * (size_t)nmax);
#pragma omp for schedule(static)
        for (int y = 0; y < ny; ++y) {
            memcpy(src, x + (size_t)y * nx, sizeof(cplx) * (size_t)nx);
            dft_rec(nx, src, 1, dst, sign);
            memcpy(x + (size_t)y * nx, dst, sizeof(cplx) * (size_t)nx);
        }
#pragma omp for schedule(static)
        for (int c = 0; c < nx; ++c) {
            for (int y = 0; y < ny; ++y) src[y] = x[(size_t)y * nx + c];
            dft_rec(ny, src, 1, dst, sign);
            for (int y = 0; y < ny; ++y) x[(size_t)y * nx + c] = dst[y];
        }
        free(src);
        free(dst);
    }
    return 0;
}

/* Angular wavenumber of DFT bin j on an n-point grid with spacing d
 * (numpy.fft.fftfreq ordering: 0, 1, ..., then the negative bins). */
static double grid_k(int j, int n, double d)
{
    int f = (j < (n + 1) / 2) ? j : j - n;
    return kTwoPi * (double)f / ((double)n * d);
}

/* Exact propagator over one slice of thickness dz (full kz, no carrier
 * factoring).  Output: [ny][nx] interleaved complex. */
int oracle_propagator(int nx, int ny, double dx, double dy, double dz,
                      double lambda, double n0, double *Hv)
{
    if (nx < 1 || ny < 1 || !(dx > 0) || !(dy > 0) || !(lambda > 0) || !(n0 > 0)) return -1;
    cplx *H = (cplx *)Hv;
    double K = kTwoPi / lambda * n0;
    for (int y = 0; y < ny; ++y) {
        double ky = grid_k(y, ny, dy);
        for (int x = 0; x < nx; ++x) {
            double kx = grid_k(x, nx, dx);
            double kz2 = K * K - kx * kx - ky * ky;
            H[(size_t)y * nx + x] = (kz2 > 0) ? cexp(I * sqrt(kz2) * dz) : 0;
        }
    }
    return 0;
}

/* Complex refractive index n = n0 + dn + i kappa (absorption for kappa > 0):
 * the same loop with the screen exp(i k0 (dn + i kappa) dz), i.e. the phase
 * exp(i k0 dn dz) times the attenuation exp(-k0 kappa dz).  kappa: [nz][ny][nx]
 * doubles; other arguments as oracle_bpm. */
int oracle_bpm_absorbing(int nx, int ny, int nz, double dx, double dy, double dz,
                         double lambda, double n0, const double *dn, const double *kappa,
                         const double *E0v, double *Eoutv, double *Iout)
{
    if (nx < 1 || ny < 1 || nz < 0 || !(dz > 0)) return -1;
    size_t M = (size_t)nx * ny;
    cplx *H = (cplx *)malloc(sizeof(cplx) * M);
    cplx *E = (cplx *)malloc(sizeof(cplx) * M);
    if (oracle_propagator(nx, ny, dx, dy, dz, lambda, n0, (double *)H) != 0) {
        free(H);
        free(E);
        return -1;
    }
    memcpy(E, E0v, sizeof(cplx) * M);
    double k0 = kTwoPi / lambda;
    for (int z = 0; z < nz; ++z) {
        oracle_dft2(nx, ny, (double *)E, -1);
        for (size_t i = 0; i < M; ++i) E[i] *= H[i];
        oracle_dft2(nx, ny, (double *)E, +1);
        const double *d_re = dn + (size_t)z * M, *d_im = kappa + (size_t)z * M;
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < (long long)M; ++i) {
            cplx e = E[i] / (double)M;
            e *= cexp(I * k0 * d_re[i] * dz) * exp(-k0 * d_im[i] * dz);
            E[i] = e;
            if (Iout) Iout[(size_t)z * M + (size_t)i] = creal(e) * creal(e) + cimag(e) * cimag(e);
        }
    }
    memcpy(Eoutv, E, sizeof(cplx) * M);
    free(H);
    free(E);
    return 0;
}

/* Reading B of the locally adapted expansion (see the header): per slice the
 * mean index step delta_z, the propagator corrected to first order in
 * delta_z, and the screen of dn - delta_z.  Arguments as oracle_bpm. */
int oracle_bpm_adaptive(int nx, int ny, int nz, double dx, double dy, double dz,
                        double lambda, double n0, const double *dn, const double *E0v,
                        double *Eoutv, double *Iout)
{
    if (nx < 1 || ny < 1 || nz < 0 || !(dz > 0) || !(dx > 0) || !(dy > 0) || !(lambda > 0) || !(n0 > 0))
        return -1;
    size_t M = (size_t)nx * ny;
    cplx *E = (cplx *)malloc(sizeof(cplx) * M);
    double *kz0 = (double *)malloc(sizeof(double) * M);   /* 0 marks a cut component */
    double k0 = kTwoPi / lambda, K = k0 * n0;
    for (int y = 0; y < ny; ++y) {
        double ky = grid_k(y, ny, dy);
        for (int x = 0; x < nx; ++x) {
            double kx = grid_k(x, nx, dx);
            double kz2 = K * K - kx * kx - ky * ky;
            kz0[(size_t)y * nx + x] = (kz2 > 0) ? sqrt(kz2) : 0.0;
        }
    }
    memcpy(E, E0v, sizeof(cplx) * M);
    for (int z = 0; z < nz; ++z) {
        const double *slice = dn + (size_t)z * M;
        double sum = 0.0;
        for (size_t i = 0; i < M; ++i) sum += slice[i];
        const double delta = sum / (double)M;
        oracle_dft2(nx, ny, (double *)E, -1);
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < (long long)M; ++i) {
            const double kz = kz0[i];
            E[i] = (kz > 0) ? E[i] * cexp(I * (kz + delta * k0 * k0 * n0 / kz) * dz) : 0;
        }
        oracle_dft2(nx, ny, (double *)E, +1);
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < (long long)M; ++i) {
            cplx e = E[i] / (double)M;
            e *= cexp(I * k0 * (slice[i] - delta) * dz);
            E[i] = e;
            if (Iout) Iout[(size_t)z * M + (size_t)i] = creal(e) * creal(e) + cimag(e) * cimag(e);
        }
    }
    memcpy(Eoutv, E, sizeof(cplx) * M);
    free(kz0);
    free(E);
    return 0;
}

/* Split-step BPM through nz slices.
 *   dn    : [nz][ny][nx] doubles, n - n0 per voxel
 *   E0    : [ny][nx] complex input field at the entrance plane
 *   Eout  : [ny][nx] complex field after the last slice (may alias E0)
 *   Iout  : [nz][ny][nx] doubles, |E|^2 after each slice's screen (nullable)
 */
int oracle_bpm(int nx, int ny, int nz, double dx, double dy, double dz,
               double lambda, double n0, const double *dn, const double *E0v,
               double *Eoutv, double *Iout)
{
    if (nx < 1 || ny < 1 || nz < 0 || !(dz > 0)) return -1;
    size_t M = (size_t)nx * ny;
    cplx *H = (cplx *)malloc(sizeof(cplx) * M);
    cplx *E = (cplx *)malloc(sizeof(cplx) * M);
    if (oracle_propagator(nx, ny, dx, dy, dz, lambda, n0, (double *)H) != 0) {
        free(H);
        free(E);
        return -1;
    }
    memcpy(E, E0v, sizeof(cplx) * M);
    double k0 = kTwoPi / lambda;
    for (int z = 0; z < nz; ++z) {
        oracle_dft2(nx, ny, (double *)E, -1);
        for (size_t i = 0; i < M; ++i) E[i] *= H[i];
        oracle_dft2(nx, ny, (double *)E, +1);
        const double *dz_slice = dn + (size_t)z * M;
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < (long long)M; ++i) {
            cplx e = E[i] / (double)M;
            e *= cexp(I * k0 * dz_slice[i] * dz);
            E[i] = e;
            if (Iout) Iout[(size_t)z * M + (size_t)i] = creal(e) * creal(e) + cimag(e) * cimag(e);
        }
    }
    memcpy(Eoutv, E, sizeof(cplx) * M);
    free(H);
    free(E);
    return 0;
}

/* Multiplexed focused input field: n_foci point emitters with phases phi_j at
 * grid points (ix_j, iy_j), each filtered by the scalar pupil |k_perp| <= k0 NA
 * (restricted to propagating waves) and defocused by exp(-i kz zf_j), so that
 * every focus forms at depth zf_j after forward propagation.  Each emitter has
 * amplitude sqrt(nx ny / n_pupil), which gives every focused field unit energy
 * sum |E|^2 = 1 before the foci are summed.  Foci at different depths are
 * synthesised one at a time and added.
 *   Eout : [ny][nx] complex, overwritten. */
/* Multiplexed focused emitters through the pupil NA_in <= |k_perp| / k0 <= NA
 * (a disk for NA_in = 0, the Bessel-beam annulus otherwise). */
static int multiplex_pupil(int nx, int ny, double dx, double dy, double lambda, double n0,
                           int n_foci, const int *ix, const int *iy, const double *phase,
                           const double *zf, double NA_in, double NA, double *Eoutv)
{
    if (nx < 1 || ny < 1 || n_foci < 0 || !(NA > 0) || !(NA_in >= 0) || !(NA_in < NA)) return -1;
    size_t M = (size_t)nx * ny;
    cplx *Eout = (cplx *)Eoutv;
    cplx *F = (cplx *)malloc(sizeof(cplx) * M);
    double k0 = kTwoPi / lambda, K = k0 * n0, kna = k0 * NA, kin = k0 * NA_in;
    long long n_pupil = 0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double kx = grid_k(x, nx, dx), ky = grid_k(y, ny, dy);
            double kp2 = kx * kx + ky * ky;
            if (kp2 >= kin * kin && kp2 <= kna * kna && K * K - kp2 > 0) ++n_pupil;
        }
    for (size_t i = 0; i < M; ++i) Eout[i] = 0;
    if (n_pupil == 0 || n_foci == 0) {
        free(F);
        return 0;
    }
    double amp = sqrt((double)M / (double)n_pupil);
    char *done = (char *)calloc((size_t)n_foci, 1);
    for (int j0 = 0; j0 < n_foci; ++j0) {
        if (done[j0]) continue;
        double zg = zf[j0];
        for (size_t i = 0; i < M; ++i) F[i] = 0;
        for (int j = j0; j < n_foci; ++j) {
            if (done[j] || zf[j] != zg) continue;
            done[j] = 1;
            if (ix[j] < 0 || ix[j] >= nx || iy[j] < 0 || iy[j] >= ny) continue;
            F[(size_t)iy[j] * nx + ix[j]] += amp * cexp(I * phase[j]);
        }
        oracle_dft2(nx, ny, (double *)F, -1);
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double kx = grid_k(x, nx, dx), ky = grid_k(y, ny, dy);
                double kp2 = kx * kx + ky * ky, kz2 = K * K - kp2;
                size_t i = (size_t)y * nx + x;
                if (kp2 >= kin * kin && kp2 <= kna * kna && kz2 > 0)
                    F[i] *= cexp(-I * sqrt(kz2) * zg);
                else
                    F[i] = 0;
            }
        oracle_dft2(nx, ny, (double *)F, +1);
        for (size_t i = 0; i < M; ++i) Eout[i] += F[i] / (double)M;
    }
    free(done);
    free(F);
    return 0;
}

int oracle_multiplex_psf(int nx, int ny, double dx, double dy, double lambda, double n0,
                         int n_foci, const int *ix, const int *iy, const double *phase,
                         const double *zf, double NA, double *Eoutv)
{
    return multiplex_pupil(nx, ny, dx, dy, lambda, n0, n_foci, ix, iy, phase, zf, 0.0, NA, Eoutv);
}

/* Bessel beams (and lattices of them, several emitters): the annular pupil
 * NA_in <= |k_perp| / k0 <= NA_out.  Arguments as oracle_multiplex_psf. */
int oracle_multiplex_annular(int nx, int ny, double dx, double dy, double lambda, double n0,
                             int n_foci, const int *ix, const int *iy, const double *phase,
                             const double *zf, double NA_in, double NA_out, double *Eoutv)
{
    return multiplex_pupil(nx, ny, dx, dy, lambda, n0, n_foci, ix, iy, phase, zf, NA_in, NA_out, Eoutv);
}

/* Cylindrical light sheet, thin along x and uniform along y: angular spectrum
 * A(kx) = exp(-(kx w0 / 2)^2) on the ky = 0 line only, w0 = lambda / (pi NA),
 * centred at x_c = (nx/2) dx, defocused by exp(-i kz zf), propagating waves
 * only, scaled so that |E|^2 = 1 at (x_c, zf) after exact propagation.
 *   Eout : [ny][nx] complex, overwritten. */
int oracle_light_sheet(int nx, int ny, double dx, double dy, double lambda, double n0,
                       double NA, double zf, double *Eoutv)
{
    if (nx < 1 || ny < 1 || !(NA > 0)) return -1;
    (void)dy;
    size_t M = (size_t)nx * ny;
    cplx *S = (cplx *)Eoutv;
    double k0 = kTwoPi / lambda, K = k0 * n0, w0 = lambda / (M_PI * NA);
    double xc = (double)(nx / 2) * dx;
    double sumA = 0;
    for (int x = 0; x < nx; ++x) {
        double kx = grid_k(x, nx, dx);
        if (K * K - kx * kx > 0) sumA += exp(-(kx * w0 / 2) * (kx * w0 / 2));
    }
    for (size_t i = 0; i < M; ++i) S[i] = 0;
    double scale = (double)M / sumA;
    for (int x = 0; x < nx; ++x) {
        double kx = grid_k(x, nx, dx), kz2 = K * K - kx * kx;
        if (!(kz2 > 0)) continue;
        double A = exp(-(kx * w0 / 2) * (kx * w0 / 2));
        S[x] = scale * A * cexp(-I * kx * xc) * cexp(-I * sqrt(kz2) * zf);
    }
    oracle_dft2(nx, ny, Eoutv, +1);
    for (size_t i = 0; i < M; ++i) S[i] /= (double)M;
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
