/*
 * FP64 CPU oracle for cascaded second-order-section (biquad) filtering.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA path is checked against.  Only tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never does.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * What it computes (paper Sec. II, Eq. general_cascaded_equation and
 * Eq. complex_second_order): a cascade y = F_K o ... o F_1 (x) where section
 * k runs the difference equation
 *
 *     y_k[n] = b0 x_k[n] + b1 x_k[n-1] + b2 x_k[n-2] - a1 y_k[n-1] - a2 y_k[n-2]
 *
 * sample by sample (the forward substitution of Sec. III,
 * Eq. recursive_equation_block_form), with x_1 = x, x_{k+1} = y_k, y = y_K.
 * Each sos row is (b0, b1, b2, a0, a1, a2); every coefficient is divided by
 * a0 first.  b0 is never factored out.
 *
 * Initial and final state use the transposed-direct-form-II convention
 * (the one scipy.signal.sosfilt uses).  The state pair (z1, z2) holds the
 * part of y[0] and y[1] that comes from samples before n = 0:
 *     z1 = b1 x[-1] + b2 x[-2] - a1 y[-1] - a2 y[-2]
 *     z2 = b2 x[-1] - a2 y[-1]
 * which are exactly the scalar corrections the paper adds to the first
 * element of the first two blocks (Sec. V-A, Eq. feedforward_block_uniform).
 * So y[0] gets +z1 and y[1] gets +z2 in place of the missing history terms,
 * and the final state is the same two sums taken at the end of the signal.
 *
 * Channels are independent.  Channel c occupies samples
 * [off_c, off_c + lengths[c]) of the packed arrays, off_c being the
 * exclusive prefix sum of lengths.  Sections k >= K[c] are ignored.
 *
 * The adjoint (oracle_sosfilt_adjoint) is the reverse-mode derivative of the
 * same loop: the transpose of the lower-triangular Toeplitz system of
 * Eq. recursive_equation_block_form, i.e. the same recurrence run backwards
 * in time.  It returns gradients with respect to x, zi and every raw sos
 * entry (including a0, through the normalisation).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* One section, forward, in place on a caller-owned FP64 buffer.
 * in[0..T) -> out[0..T).  c = (b0,b1,b2,a1,a2) normalised.  zi/zf are
 * 2-vectors (zf may alias nothing else). */
static void section_forward(const double *in, double *out, int64_t T,
                            const double c[5], const double zi[2], double zf[2])
{
    const double b0 = c[0], b1 = c[1], b2 = c[2], a1 = c[3], a2 = c[4];
    for (int64_t n = 0; n < T; ++n) {
        double acc = b0 * in[n];
        if (n >= 1) acc += b1 * in[n - 1] - a1 * out[n - 1];
        if (n >= 2) acc += b2 * in[n - 2] - a2 * out[n - 2];
        if (n == 0) acc += zi[0];
        if (n == 1) acc += zi[1];
        out[n] = acc;
    }
    /* final state: the same history sums, evaluated one and two samples past
     * the end; history that does not exist comes from zi */
    double z1 = 0.0, z2 = 0.0;
    if (T >= 1) {
        z1 += b1 * in[T - 1] - a1 * out[T - 1];
        z2 += b2 * in[T - 1] - a2 * out[T - 1];
    }
    if (T >= 2) z1 += b2 * in[T - 2] - a2 * out[T - 2];
    if (T == 1) z1 += zi[1];
    if (T == 0) { z1 = zi[0]; z2 = zi[1]; }
    zf[0] = z1;
    zf[1] = z2;
}

static void normalise(const double *row, double c[5])
{
    const double a0 = row[3];
    c[0] = row[0] / a0;
    c[1] = row[1] / a0;
    c[2] = row[2] / a0;
    c[3] = row[4] / a0;
    c[4] = row[5] / a0;
}

/* returns 0 on success, -1 on a bad argument */
int oracle_sosfilt(const double *x, const double *sos, const int32_t *K,
                   int32_t n_channels, int32_t kmax, const int64_t *lengths,
                   const double *zi, double *y, double *zf)
{
    if (n_channels < 0 || kmax < 1) return -1;
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_channels + 1));
    if (!off) return -1;
    off[0] = 0;
    for (int32_t c = 0; c < n_channels; ++c) {
        if (lengths[c] < 0 || K[c] < 0 || K[c] > kmax) { free(off); return -1; }
        off[c + 1] = off[c] + lengths[c];
    }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int32_t c = 0; c < n_channels; ++c) {
        const int64_t T = lengths[c];
        double *buf = (double *)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
        if (!buf) { bad |= 1; continue; }
        const double *src = x + off[c];
        double *dst = y + off[c];
        /* ping-pong between the output slice and a scratch buffer so that the
         * last section lands in y */
        const double *cur = src;
        for (int32_t k = 0; k < K[c]; ++k) {
            double cf[5];
            normalise(sos + ((int64_t)c * kmax + k) * 6, cf);
            const double zero2[2] = {0.0, 0.0};
            const double *z0 = zi ? zi + ((int64_t)c * kmax + k) * 2 : zero2;
            double zfk[2];
            double *out = ((K[c] - 1 - k) % 2 == 0) ? dst : buf;
            section_forward(cur, out, T, cf, z0, zfk);
            if (zf) {
                zf[((int64_t)c * kmax + k) * 2 + 0] = zfk[0];
                zf[((int64_t)c * kmax + k) * 2 + 1] = zfk[1];
            }
            cur = out;
        }
        if (K[c] == 0) memcpy(dst, src, sizeof(double) * (size_t)T);
        if (zf) {
            for (int32_t k = K[c]; k < kmax; ++k) {
                zf[((int64_t)c * kmax + k) * 2 + 0] = 0.0;
                zf[((int64_t)c * kmax + k) * 2 + 1] = 0.0;
            }
        }
        free(buf);
    }
    free(off);
    return bad ? -1 : 0;
}

/* Reverse mode of section_forward.  Given the section's input/output and the
 * incoming adjoints g_out (dL/dout) and g_zf (dL/dzf), produce dL/din,
 * dL/dc (normalised coefficients) and dL/dzi.  Each statement of the forward
 * loop is differentiated in reverse order. */
static void section_adjoint(const double *in, const double *out, int64_t T,
                            const double c[5], const double g_zf[2],
                            double *g_out /* modified in place */,
                            double *g_in, double g_c[5], double g_zi[2])
{
    const double b0 = c[0], b1 = c[1], b2 = c[2], a1 = c[3], a2 = c[4];
    for (int i = 0; i < 5; ++i) g_c[i] = 0.0;
    g_zi[0] = 0.0;
    g_zi[1] = 0.0;
    for (int64_t n = 0; n < T; ++n) g_in[n] = 0.0;

    /* final state */
    const double gz1 = g_zf[0], gz2 = g_zf[1];
    if (T == 0) { g_zi[0] += gz1; g_zi[1] += gz2; return; }
    if (T == 1) g_zi[1] += gz1;
    if (T >= 2) {
        g_c[2] += gz1 * in[T - 2];
        g_in[T - 2] += gz1 * b2;
        g_c[4] -= gz1 * out[T - 2];
        g_out[T - 2] -= gz1 * a2;
    }
    /* T >= 1 */
    g_c[1] += gz1 * in[T - 1];
    g_in[T - 1] += gz1 * b1;
    g_c[3] -= gz1 * out[T - 1];
    g_out[T - 1] -= gz1 * a1;
    g_c[2] += gz2 * in[T - 1];
    g_in[T - 1] += gz2 * b2;
    g_c[4] -= gz2 * out[T - 1];
    g_out[T - 1] -= gz2 * a2;

    /* the recurrence, last sample first */
    for (int64_t n = T - 1; n >= 0; --n) {
        const double g = g_out[n]; /* complete: later samples already added */
        if (n == 1) g_zi[1] += g;
        if (n == 0) g_zi[0] += g;
        if (n >= 2) {
            g_c[2] += g * in[n - 2];
            g_in[n - 2] += g * b2;
            g_c[4] -= g * out[n - 2];
            g_out[n - 2] -= g * a2;
        }
        if (n >= 1) {
            g_c[1] += g * in[n - 1];
            g_in[n - 1] += g * b1;
            g_c[3] -= g * out[n - 1];
            g_out[n - 1] -= g * a1;
        }
        g_c[0] += g * in[n];
        g_in[n] += g * b0;
    }
}

/* Gradients of a scalar loss L(y, zf) given dL/dy (g_y, packed like y) and
 * dL/dzf (g_zf, [C][kmax][2], may be NULL = zero).
 * Outputs: g_x (packed like x), g_sos ([C][kmax][6], raw rows incl. a0),
 * g_zi ([C][kmax][2]).  Any output pointer may be NULL. */
int oracle_sosfilt_adjoint(const double *x, const double *sos, const int32_t *K,
                           int32_t n_channels, int32_t kmax, const int64_t *lengths,
                           const double *zi, const double *g_y, const double *g_zf,
                           double *g_x, double *g_sos, double *g_zi)
{
    if (n_channels < 0 || kmax < 1) return -1;
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_channels + 1));
    if (!off) return -1;
    off[0] = 0;
    for (int32_t c = 0; c < n_channels; ++c) {
        if (lengths[c] < 0 || K[c] < 0 || K[c] > kmax) { free(off); return -1; }
        off[c + 1] = off[c] + lengths[c];
    }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int32_t c = 0; c < n_channels; ++c) {
        const int64_t T = lengths[c];
        const int32_t Kc = K[c];
        const size_t Tn = (size_t)(T > 0 ? T : 1);
        /* sig[k] = input of section k; sig[Kc] = final output */
        double *sig = (double *)malloc(sizeof(double) * Tn * (size_t)(Kc + 1));
        double *ga = (double *)malloc(sizeof(double) * Tn);
        double *gb = (double *)malloc(sizeof(double) * Tn);
        if (!sig || !ga || !gb) { bad |= 1; free(sig); free(ga); free(gb); continue; }
        for (int64_t n = 0; n < T; ++n) sig[n] = x[off[c] + n];
        double cfk[5];
        for (int32_t k = 0; k < Kc; ++k) {
            normalise(sos + ((int64_t)c * kmax + k) * 6, cfk);
            const double zero2[2] = {0.0, 0.0};
            const double *z0 = zi ? zi + ((int64_t)c * kmax + k) * 2 : zero2;
            double zfk[2];
            section_forward(sig + (size_t)k * Tn, sig + (size_t)(k + 1) * Tn, T, cfk, z0, zfk);
        }
        /* ga = dL/d(output of the current section) */
        for (int64_t n = 0; n < T; ++n) ga[n] = g_y ? g_y[off[c] + n] : 0.0;
        for (int32_t k = Kc - 1; k >= 0; --k) {
            double c5[5];
            normalise(sos + ((int64_t)c * kmax + k) * 6, c5);
            const double zero2[2] = {0.0, 0.0};
            const double *gzf = g_zf ? g_zf + ((int64_t)c * kmax + k) * 2 : zero2;
            double gc[5], gzi[2];
            section_adjoint(sig + (size_t)k * Tn, sig + (size_t)(k + 1) * Tn, T, c5, gzf,
                            ga, gb, gc, gzi);
            if (g_zi) {
                g_zi[((int64_t)c * kmax + k) * 2 + 0] = gzi[0];
                g_zi[((int64_t)c * kmax + k) * 2 + 1] = gzi[1];
            }
            if (g_sos) {
                const double *row = sos + ((int64_t)c * kmax + k) * 6;
                double *gr = g_sos + ((int64_t)c * kmax + k) * 6;
                const double a0 = row[3];
                /* c5 = (b0,b1,b2,a1,a2)/a0 */
                gr[0] = gc[0] / a0;
                gr[1] = gc[1] / a0;
                gr[2] = gc[2] / a0;
                gr[4] = gc[3] / a0;
                gr[5] = gc[4] / a0;
                gr[3] = -(gc[0] * c5[0] + gc[1] * c5[1] + gc[2] * c5[2] +
                          gc[3] * c5[3] + gc[4] * c5[4]) / a0;
            }
            double *t = ga; ga = gb; gb = t; /* input adjoint feeds the previous section */
        }
        if (g_x)
            for (int64_t n = 0; n < T; ++n) g_x[off[c] + n] = ga[n];
        for (int32_t k = Kc; k < kmax; ++k) {
            if (g_zi) {
                g_zi[((int64_t)c * kmax + k) * 2 + 0] = 0.0;
                g_zi[((int64_t)c * kmax + k) * 2 + 1] = 0.0;
            }
            if (g_sos)
                for (int j = 0; j < 6; ++j) g_sos[((int64_t)c * kmax + k) * 6 + j] = 0.0;
        }
        free(sig); free(ga); free(gb);
    }
    free(off);
    return bad ? -1 : 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
