/*
 * cwo_oracle.c -- plain, slow, FP64 CPU oracle for FFT-based scalar diffraction as defined in
 * Shimobaba et al., "Computational wave optics library for C++: CWO++ library":
 *   - Fresnel diffraction, convolution form  (Section "Fresnel diffraction (convolution form)",
 *     Eqs. fre_conv, fresnel_conv, fre_conv_prop, fre_conv_fft, fre_conv_prop_d)
 *   - angular spectrum method                (Section "Angular spectrum method", Eqs. ang1-ang3)
 *   - zero padding N -> 2N and crop of the exact N x N area (Section "Summary of diffraction
 *     calculation", Table "Classification of diffraction calculation")
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it. It shares no code, header, table or constant with the CUDA path:
 * every formula below is written out from the paper in its own notation, in double precision,
 * without blocking, fusion or reordering beyond what the definitions state.
 *
 * Conventions (the paper leaves these unstated; the readings are listed in the design notes):
 *   - forward DFT   X[k] = sum_n x[n] exp(-2 pi i k n / P)      (unscaled, FFTW/CUFFT sign)
 *   - inverse DFT   x[n] = (1/P) sum_k X[k] exp(+2 pi i k n / P)
 *   - the N x N input sits in the top-left block of the P x P grid; the crop keeps that block
 *   - frequency of bin k on the padded grid: f = kt / (P * pitch), kt = k (k < P/2) else k - P
 *   - evanescent components of the angular spectrum transfer function are set to zero
 *   - Fresnel impulse response sample at grid index i has displacement d = i (i < P/2) else i - P
 *   - Fresnel coefficient includes the area element dx*dy unless ORC_LITERAL_SCALE is given
 *
 * Arrays are row-major [ny][nx] of interleaved (re, im) doubles, i.e. C99 double complex.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846264338327950288

/* flags */
#define ORC_ADJOINT       1u  /* use conj(H) and conj(C): the adjoint of the linear map        */
#define ORC_NO_PAD        2u  /* circular convolution on the N grid (test mode, no padding)    */
#define ORC_FULL_OUTPUT   4u  /* return the whole P x P grid instead of the N x N crop         */
#define ORC_LITERAL_SCALE 8u  /* Fresnel: drop the dx*dy area element from the coefficient     */

/* diffraction types */
#define ORC_ANGULAR      0
#define ORC_FRESNEL_CONV 1

/* status */
#define ORC_OK           0
#define ORC_EINVAL      -1
#define ORC_ENOMEM      -2

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops that follow (timing only: each row or column transform is
 * computed by one thread in the same order whatever the count, so results do not depend on it). */
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static int is_pow2(long n) { return n >= 1 && (n & (n - 1)) == 0; }

/* Signed bin index on a grid of n points: k for k < n/2, k - n otherwise.  Bin n/2 (Nyquist)
 * maps to -n/2. */
static long signed_bin(long k, long n) { return (k < n / 2) ? k : k - n; }

/* ---------------------------------------------------------------------------------------------
 * Direct DFT, straight from the definition: X[k] = sum_j x[j] exp(sign * 2 pi i j k / n).
 * The product j*k is reduced modulo n in integer arithmetic before it becomes an angle.
 * ------------------------------------------------------------------------------------------- */
void orc_dft(const cplx* x, cplx* X, long n, int sign) {
    for (long k = 0; k < n; ++k) {
        cplx acc = 0.0;
        for (long j = 0; j < n; ++j) {
            long jk = (j * k) % n;
            double ang = (double)sign * 2.0 * ORC_PI * (double)jk / (double)n;
            acc += x[j] * cexp(I * ang);
        }
        X[k] = acc;
    }
}

/* ---------------------------------------------------------------------------------------------
 * Textbook iterative radix-2 Cooley-Tukey FFT (decimation in time), in place, unscaled:
 * bit-reversal permutation, then log2(n) layers of butterflies.  w holds exp(sign 2 pi i j / n)
 * for j < n/2, each entry evaluated on its own with cexp.
 * ------------------------------------------------------------------------------------------- */
static void fft_table(cplx* w, long n, int sign) {
    for (long j = 0; j < n / 2; ++j) w[j] = cexp(I * ((double)sign * 2.0 * ORC_PI * (double)j / (double)n));
}

static void fft_with_table(cplx* a, long n, const cplx* w) {
    for (long i = 1, j = 0; i < n; ++i) {
        long bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (long len = 2; len <= n; len <<= 1) {
        long half = len / 2, step = n / len;
        for (long i = 0; i < n; i += len) {
            for (long j = 0; j < half; ++j) {
                cplx u = a[i + j];
                cplx v = a[i + j + half] * w[j * step];
                a[i + j] = u + v;
                a[i + j + half] = u - v;
            }
        }
    }
}

int orc_fft(cplx* a, long n, int sign) {
    if (!is_pow2(n)) return ORC_EINVAL;
    if (n == 1) return ORC_OK;
    cplx* w = malloc(sizeof(cplx) * (size_t)(n / 2));
    if (!w) return ORC_ENOMEM;
    fft_table(w, n, sign);
    fft_with_table(a, n, w);
    free(w);
    return ORC_OK;
}

/* 2-D FFT of a row-major [rows][cols] array: 1-D FFT of every row, then of every column. */
int orc_fft2(cplx* a, long rows, long cols, int sign) {
    if (!is_pow2(rows) || !is_pow2(cols)) return ORC_EINVAL;
    cplx* wr = malloc(sizeof(cplx) * (size_t)(cols / 2 + 1));
    cplx* wc = malloc(sizeof(cplx) * (size_t)(rows / 2 + 1));
    if (!wr || !wc) { free(wr); free(wc); return ORC_ENOMEM; }
    fft_table(wr, cols, sign);
    fft_table(wc, rows, sign);
    if (cols > 1) {
        #pragma omp parallel for schedule(static)
        for (long r = 0; r < rows; ++r) fft_with_table(a + r * cols, cols, wr);
    }
    if (rows > 1) {
        int fail = 0;
        #pragma omp parallel
        {
            cplx* col = malloc(sizeof(cplx) * (size_t)rows);
            if (!col) {
                #pragma omp atomic write
                fail = 1;
            } else {
                #pragma omp for schedule(static)
                for (long c = 0; c < cols; ++c) {
                    for (long r = 0; r < rows; ++r) col[r] = a[r * cols + c];
                    fft_with_table(col, rows, wc);
                    for (long r = 0; r < rows; ++r) a[r * cols + c] = col[r];
                }
                free(col);
            }
        }
        if (fail) { free(wr); free(wc); return ORC_ENOMEM; }
    }
    free(wr); free(wc);
    return ORC_OK;
}

/* ---------------------------------------------------------------------------------------------
 * Angular spectrum transfer function, Eq. ang2:
 *     H_A(fx, fy) = exp(i z sqrt(k^2 - 4 pi^2 (fx^2 + fy^2))),   k = 2 pi / lambda,
 * sampled at fx = kt_x / (px dx), fy = kt_y / (py dy).  Where the radicand is negative
 * (evanescent waves) H_A = 0.
 * ------------------------------------------------------------------------------------------- */
static cplx asm_transfer(long kx, long ky, long px, long py, double dx, double dy, double lambda, double z) {
    double fx = (double)signed_bin(kx, px) / ((double)px * dx);
    double fy = (double)signed_bin(ky, py) / ((double)py * dy);
    double k = 2.0 * ORC_PI / lambda;
    double rad = k * k - 4.0 * ORC_PI * ORC_PI * (fx * fx + fy * fy);
    if (rad < 0.0) return 0.0;
    return cexp(I * (z * sqrt(rad)));
}

/* Fill H[py][px] with the angular spectrum transfer function (exposed for tests). */
void orc_asm_transfer(cplx* H, long px, long py, double dx, double dy, double lambda, double z) {
    for (long ky = 0; ky < py; ++ky)
        for (long kx = 0; kx < px; ++kx)
            H[ky * px + kx] = asm_transfer(kx, ky, px, py, dx, dy, lambda, z);
}

/* Fresnel impulse response, Eq. fre_conv_prop_d: h_F(m, n) = exp(i pi ((m dx)^2 + (n dy)^2) / (lambda z)). */
static cplx fresnel_impulse(long m, long n, double dx, double dy, double lambda, double z) {
    double x = (double)m * dx, y = (double)n * dy;
    return cexp(I * (ORC_PI * (x * x + y * y) / (lambda * z)));
}

/* Fresnel coefficient, Eq. fre_conv_fft: exp(i 2 pi z / lambda) / (i lambda z), times the area
 * element dx*dy of the discretised integral of Eq. fre_conv unless ORC_LITERAL_SCALE. */
static cplx fresnel_coeff(double dx, double dy, double lambda, double z, unsigned flags) {
    cplx c = cexp(I * (2.0 * ORC_PI * z / lambda)) / (I * lambda * z);
    if (!(flags & ORC_LITERAL_SCALE)) c *= dx * dy;
    return c;
}

/* ---------------------------------------------------------------------------------------------
 * FFT-based propagation, exactly the steps of the paper:
 *   1. expand the Nx x Ny source into the top-left corner of a 2Nx x 2Ny grid of zeros
 *   2. FFT
 *   3. multiply by the transfer function
 *        ASM (Eq. ang3):      H_A of Eq. ang2
 *        Fresnel (Eq. fre_conv_fft): C * FFT[h_F], h_F sampled on the padded grid (the third FFT)
 *   4. inverse FFT (scaled by 1/(px py))
 *   5. extract the Nx x Ny area.
 * With ORC_ADJOINT the transfer function (and C) is conjugated.
 * u1: [ny][nx];  u2: [ny][nx], or [py][px] with ORC_FULL_OUTPUT.
 * ------------------------------------------------------------------------------------------- */
int orc_propagate(const cplx* u1, cplx* u2, long nx, long ny, double dx, double dy,
                  double lambda, double z, int type, unsigned flags) {
    if (!is_pow2(nx) || !is_pow2(ny) || nx < 2 || ny < 2) return ORC_EINVAL;
    if (!(dx > 0) || !(dy > 0) || !(lambda > 0)) return ORC_EINVAL;
    if (type != ORC_ANGULAR && type != ORC_FRESNEL_CONV) return ORC_EINVAL;
    if (type == ORC_FRESNEL_CONV && z == 0.0) return ORC_EINVAL;
    long px = (flags & ORC_NO_PAD) ? nx : 2 * nx;
    long py = (flags & ORC_NO_PAD) ? ny : 2 * ny;
    int conj_h = (flags & ORC_ADJOINT) != 0;

    cplx* U = calloc((size_t)(px * py), sizeof(cplx));
    if (!U) return ORC_ENOMEM;
    for (long y = 0; y < ny; ++y)                                   /* step 1: expand */
        for (long x = 0; x < nx; ++x) U[y * px + x] = u1[y * nx + x];
    int st = orc_fft2(U, py, px, -1);                               /* step 2: FFT */
    if (st) { free(U); return st; }

    if (type == ORC_ANGULAR) {                                      /* step 3 (ASM) */
        #pragma omp parallel for schedule(static)
        for (long ky = 0; ky < py; ++ky)
            for (long kx = 0; kx < px; ++kx) {
                cplx H = asm_transfer(kx, ky, px, py, dx, dy, lambda, z);
                U[ky * px + kx] *= conj_h ? conj(H) : H;
            }
    } else {                                                        /* step 3 (Fresnel) */
        cplx* h = malloc(sizeof(cplx) * (size_t)(px * py));
        if (!h) { free(U); return ORC_ENOMEM; }
        #pragma omp parallel for schedule(static)
        for (long iy = 0; iy < py; ++iy)
            for (long ix = 0; ix < px; ++ix)
                h[iy * px + ix] = fresnel_impulse(signed_bin(ix, px), signed_bin(iy, py), dx, dy, lambda, z);
        st = orc_fft2(h, py, px, -1);
        if (st) { free(h); free(U); return st; }
        cplx C = fresnel_coeff(dx, dy, lambda, z, flags);
        #pragma omp parallel for schedule(static)
        for (long i = 0; i < px * py; ++i) {
            cplx H = C * h[i];
            U[i] *= conj_h ? conj(H) : H;
        }
        free(h);
    }

    st = orc_fft2(U, py, px, +1);                                   /* step 4: inverse FFT */
    if (st) { free(U); return st; }
    double s = 1.0 / ((double)px * (double)py);
    if (flags & ORC_FULL_OUTPUT) {
        for (long i = 0; i < px * py; ++i) u2[i] = U[i] * s;
    } else {                                                        /* step 5: extract */
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) u2[y * nx + x] = U[y * px + x] * s;
    }
    free(U);
    return ORC_OK;
}

/* ---------------------------------------------------------------------------------------------
 * Brute-force direct sums (tiny grids only).  With the source in the top-left N x N block of a
 * 2N x 2N grid and the crop keeping the same block, every index difference d = m2 - m1 lies in
 * [-(N-1), N-1], so the circular convolution computed by the padded FFT method equals this
 * linear convolution exactly.
 *
 * Fresnel (Eqs. fre_conv and fre_conv_prop_d, discretised):
 *     u2[n2][m2] = C * sum_{m1, n1} u1[n1][m1] * h_F(m2 - m1, n2 - n1)
 * ASM (Eq. ang3 written as a convolution):
 *     u2[n2][m2] = sum_{m1, n1} u1[n1][m1] * h_A(m2 - m1, n2 - n1),
 *     h_A(d, e) = (1/(px py)) sum_{kx, ky} H_A(kx, ky) exp(+2 pi i (kx d / px + ky e / py))
 * ------------------------------------------------------------------------------------------- */
int orc_propagate_direct(const cplx* u1, cplx* u2, long nx, long ny, double dx, double dy,
                         double lambda, double z, int type, unsigned flags) {
    if (nx < 1 || ny < 1 || nx > 64 || ny > 64) return ORC_EINVAL;
    if (!(dx > 0) || !(dy > 0) || !(lambda > 0)) return ORC_EINVAL;
    if (type == ORC_FRESNEL_CONV && z == 0.0) return ORC_EINVAL;
    if (flags & (ORC_NO_PAD | ORC_FULL_OUTPUT)) return ORC_EINVAL;
    int conj_h = (flags & ORC_ADJOINT) != 0;
    long wx = 2 * nx - 1, wy = 2 * ny - 1;          /* displacements -(N-1) .. N-1 */
    cplx* ker = malloc(sizeof(cplx) * (size_t)(wx * wy));
    if (!ker) return ORC_ENOMEM;

    if (type == ORC_FRESNEL_CONV) {
        cplx C = fresnel_coeff(dx, dy, lambda, z, flags);
        for (long e = -(ny - 1); e <= ny - 1; ++e)
            for (long d = -(nx - 1); d <= nx - 1; ++d) {
                cplx v = C * fresnel_impulse(d, e, dx, dy, lambda, z);
                ker[(e + ny - 1) * wx + (d + nx - 1)] = conj_h ? conj(v) : v;
            }
    } else if (type == ORC_ANGULAR) {
        long px = 2 * nx, py = 2 * ny;
        for (long e = -(ny - 1); e <= ny - 1; ++e)
            for (long d = -(nx - 1); d <= nx - 1; ++d) {
                cplx acc = 0.0;
                for (long ky = 0; ky < py; ++ky)
                    for (long kx = 0; kx < px; ++kx) {
                        cplx H = asm_transfer(kx, ky, px, py, dx, dy, lambda, z);
                        if (conj_h) H = conj(H);
                        long ax = ((kx * (d + px)) % px), ay = ((ky * (e + py)) % py);
                        double ang = 2.0 * ORC_PI * ((double)ax / (double)px + (double)ay / (double)py);
                        acc += H * cexp(I * ang);
                    }
                ker[(e + ny - 1) * wx + (d + nx - 1)] = acc / ((double)px * (double)py);
            }
    } else {
        free(ker);
        return ORC_EINVAL;
    }

    for (long n2 = 0; n2 < ny; ++n2)
        for (long m2 = 0; m2 < nx; ++m2) {
            cplx acc = 0.0;
            for (long n1 = 0; n1 < ny; ++n1)
                for (long m1 = 0; m1 < nx; ++m1)
                    acc += u1[n1 * nx + m1] * ker[(n2 - n1 + ny - 1) * wx + (m2 - m1 + nx - 1)];
            u2[n2 * nx + m2] = acc;
        }
    free(ker);
    return ORC_OK;
}
