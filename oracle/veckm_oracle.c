/*
 * FP64 CPU oracle for the local event encoder and flow head of
 * "A Real-Time Event-Based Normal Flow Estimator" (arXiv 2504.19417).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with
 * the CUDA library: phases here come from libm sin/cos on FP64 arguments,
 * never from tables.
 *
 * Functions and the passages they follow:
 *   oracle_encode_direct  Eq. (emb) of Section 2.2.1 written out: for each
 *                         requested event k, the mean over every slice event
 *                         j in its spatial window (|x_j-x_k| <= dx and
 *                         |y_j-y_k| <= dy, Eq. 1, no temporal window) of
 *                         exp(i[(t_j-t_k)/dt T + (x_j-x_k)/dx X + (y_j-y_k)/dy Y]).
 *                         This is the adjacency-matrix (O(N^2)) form.
 *   oracle_encode_pooled  Algorithm 1 in its own order: PixelEmbed/PixelCount
 *                         accumulation of the temporal phase (its first loop),
 *                         then for each requested event the window loop with
 *                         the precomputed spatial phase, the conjugate
 *                         temporal phase and the division by the window
 *                         count (its second loop; Eq. 16-17).
 *   oracle_mlp            The two-layer perceptron of Eq. 6:
 *                         flow = W2 ReLU(W1 [Re emb; Im emb] + b1) + b2.
 *   oracle_kde_query      Lemma 1 of Section 2.2.1: Re((1/D) sum_d emb[d]
 *                         conj(phi_d(q))), the kernel density read back from
 *                         an encoding at a query offset q.
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes):
 *   - Times are integer microseconds measured from a caller-given slice start
 *     t_ref; t_j - t_k and t_k - t_ref are exact integers before conversion
 *     to double.  Algorithm 1 uses absolute t_k/dt; the result is the same in
 *     exact arithmetic because only time differences survive.
 *   - Pixels outside [0,W) x [0,H) hold no events and contribute nothing.
 *   - The normaliser is the window count, which includes the event itself.
 *   - Output layout: emb[k][0..D-1] real parts, emb[k][D..2D-1] imaginary
 *     parts; the perceptron input is that same row.
 *
 * Status codes: 0 ok, -1 bad argument, -2 out of memory, -4 an event or
 * index out of range.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ERANGE (-4)

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static int check_events(const int16_t *x, const int16_t *y, const uint32_t *t, int64_t n,
                        uint32_t t_ref, int32_t W, int32_t H) {
    for (int64_t j = 0; j < n; ++j) {
        if (x[j] < 0 || x[j] >= W || y[j] < 0 || y[j] >= H) return ORC_ERANGE;
        if (t[j] < t_ref) return ORC_ERANGE;
    }
    return ORC_OK;
}

static int check_common(const int16_t *x, const int16_t *y, const uint32_t *t, int64_t n,
                        uint32_t t_ref, const int64_t *K, int64_t nK, int32_t W, int32_t H,
                        int32_t D, int32_t dx, int32_t dy, double dt) {
    if (n < 0 || nK < 0 || W <= 0 || H <= 0 || D <= 0 || dx < 0 || dy < 0 || !(dt > 0.0))
        return ORC_EINVAL;
    if (n > 0 && (!x || !y || !t)) return ORC_EINVAL;
    int rc = check_events(x, y, t, n, t_ref, W, H);
    if (rc) return rc;
    if (K) {
        for (int64_t i = 0; i < nK; ++i)
            if (K[i] < 0 || K[i] >= n) return ORC_ERANGE;
    } else if (nK != n) {
        return ORC_EINVAL;
    }
    return ORC_OK;
}

/* Eq. (emb): direct sum over the window, one requested event at a time. */
int oracle_encode_direct(const int16_t *x, const int16_t *y, const uint32_t *t, int64_t n,
                         uint32_t t_ref, const int64_t *K, int64_t nK, int32_t W, int32_t H,
                         int32_t D, int32_t dx, int32_t dy, double dt_us, const double *T,
                         const double *X, const double *Y, double *emb, int64_t *count) {
    int rc = check_common(x, y, t, n, t_ref, K, nK, W, H, D, dx, dy, dt_us);
    if (rc) return rc;
    if (nK > 0 && (!T || !X || !Y || !emb)) return ORC_EINVAL;
    (void)t_ref;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nK; ++i) {
        const int64_t k = K ? K[i] : i;
        double *re = emb + i * 2 * (int64_t)D, *im = re + D;
        for (int32_t d = 0; d < D; ++d) re[d] = im[d] = 0.0;
        int64_t cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            const int32_t ex = (int32_t)x[j] - x[k], ey = (int32_t)y[j] - y[k];
            if (ex < -dx || ex > dx || ey < -dy || ey > dy) continue;
            ++cnt;
            const double ut = (double)((int64_t)t[j] - (int64_t)t[k]) / dt_us;
            const double ux = dx > 0 ? (double)ex / dx : 0.0;
            const double uy = dy > 0 ? (double)ey / dy : 0.0;
            for (int32_t d = 0; d < D; ++d) {
                const double a = ut * T[d] + ux * X[d] + uy * Y[d];
                re[d] += cos(a);
                im[d] += sin(a);
            }
        }
        for (int32_t d = 0; d < D; ++d) {
            re[d] /= (double)cnt;
            im[d] /= (double)cnt;
        }
        if (count) count[i] = cnt;
    }
    return ORC_OK;
}

/* Algorithm 1: PixelEmbed / PixelCount, then the per-event window loop. */
int oracle_encode_pooled(const int16_t *x, const int16_t *y, const uint32_t *t, int64_t n,
                         uint32_t t_ref, const int64_t *K, int64_t nK, int32_t W, int32_t H,
                         int32_t D, int32_t dx, int32_t dy, double dt_us, const double *T,
                         const double *X, const double *Y, double *emb, int64_t *count) {
    int rc = check_common(x, y, t, n, t_ref, K, nK, W, H, D, dx, dy, dt_us);
    if (rc) return rc;
    if (nK == 0) return ORC_OK;
    if (!T || !X || !Y || !emb) return ORC_EINVAL;
    const int64_t P = (int64_t)W * H;
    /* PixelEmbed[x, y, :] as separate real and imaginary planes, pixel-major. */
    double *pe_re = (double *)calloc((size_t)(P * D), sizeof(double));
    double *pe_im = (double *)calloc((size_t)(P * D), sizeof(double));
    int64_t *pc = (int64_t *)calloc((size_t)P, sizeof(int64_t));
    const int32_t nwx = 2 * dx + 1, nwy = 2 * dy + 1;
    /* the "precomputed" spatial factors exp(i dx/delta_x X), exp(i dy/delta_y Y) */
    double *sx_re = (double *)malloc(sizeof(double) * (size_t)nwx * D);
    double *sx_im = (double *)malloc(sizeof(double) * (size_t)nwx * D);
    double *sy_re = (double *)malloc(sizeof(double) * (size_t)nwy * D);
    double *sy_im = (double *)malloc(sizeof(double) * (size_t)nwy * D);
    if (!pe_re || !pe_im || !pc || !sx_re || !sx_im || !sy_re || !sy_im) {
        free(pe_re); free(pe_im); free(pc); free(sx_re); free(sx_im); free(sy_re); free(sy_im);
        return ORC_ENOMEM;
    }
    /* first loop: accumulate exp(i t_k/dt T) and the count at each event's pixel */
    for (int64_t k = 0; k < n; ++k) {
        const int64_t p = (int64_t)x[k] * H + y[k];
        const double ut = (double)((int64_t)t[k] - (int64_t)t_ref) / dt_us;
        double *r = pe_re + p * D, *m = pe_im + p * D;
        for (int32_t d = 0; d < D; ++d) {
            r[d] += cos(ut * T[d]);
            m[d] += sin(ut * T[d]);
        }
        pc[p] += 1;
    }
    for (int32_t a = -dx; a <= dx; ++a)
        for (int32_t d = 0; d < D; ++d) {
            const double ang = (dx > 0 ? (double)a / dx : 0.0) * X[d];
            sx_re[(a + dx) * D + d] = cos(ang);
            sx_im[(a + dx) * D + d] = sin(ang);
        }
    for (int32_t b = -dy; b <= dy; ++b)
        for (int32_t d = 0; d < D; ++d) {
            const double ang = (dy > 0 ? (double)b / dy : 0.0) * Y[d];
            sy_re[(b + dy) * D + d] = cos(ang);
            sy_im[(b + dy) * D + d] = sin(ang);
        }
    /* second loop: window sum with the spatial factors, conjugate phase, 1/count */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nK; ++i) {
        const int64_t k = K ? K[i] : i;
        double *re = emb + i * 2 * (int64_t)D, *im = re + D;
        for (int32_t d = 0; d < D; ++d) re[d] = im[d] = 0.0;
        int64_t cnt = 0;
        for (int32_t a = -dx; a <= dx; ++a) {
            const int32_t px = x[k] + a;
            if (px < 0 || px >= W) continue;
            for (int32_t b = -dy; b <= dy; ++b) {
                const int32_t py = y[k] + b;
                if (py < 0 || py >= H) continue;
                const int64_t p = (int64_t)px * H + py;
                cnt += pc[p];
                if (pc[p] == 0) continue;
                const double *r = pe_re + p * D, *m = pe_im + p * D;
                const double *xr = sx_re + (a + dx) * D, *xi = sx_im + (a + dx) * D;
                const double *yr = sy_re + (b + dy) * D, *yi = sy_im + (b + dy) * D;
                for (int32_t d = 0; d < D; ++d) {
                    const double sr = xr[d] * yr[d] - xi[d] * yi[d];
                    const double si = xr[d] * yi[d] + xi[d] * yr[d];
                    re[d] += r[d] * sr - m[d] * si;
                    im[d] += r[d] * si + m[d] * sr;
                }
            }
        }
        const double ut = (double)((int64_t)t[k] - (int64_t)t_ref) / dt_us;
        for (int32_t d = 0; d < D; ++d) {
            const double cr = cos(ut * T[d]), ci = -sin(ut * T[d]);
            const double vr = re[d] * cr - im[d] * ci, vi = re[d] * ci + im[d] * cr;
            re[d] = vr / (double)cnt;
            im[d] = vi / (double)cnt;
        }
        if (count) count[i] = cnt;
    }
    free(pe_re); free(pe_im); free(pc); free(sx_re); free(sx_im); free(sy_re); free(sy_im);
    return ORC_OK;
}

/* Eq. 6 with the width and activation fixed by the workload definition:
 * flow = W2 ReLU(W1 e + b1) + b2, e = [Re emb; Im emb] (row of length 2D). */
int oracle_mlp(const double *emb, int64_t nK, int32_t D, int32_t hidden, const float *W1,
               const float *b1, const float *W2, const float *b2, double *flow) {
    if (nK < 0 || D <= 0 || hidden <= 0) return ORC_EINVAL;
    if (nK == 0) return ORC_OK;
    if (!emb || !W1 || !b1 || !W2 || !b2 || !flow) return ORC_EINVAL;
    const int32_t in = 2 * D;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nK; ++i) {
        const double *e = emb + i * in;
        double o0 = (double)b2[0], o1 = (double)b2[1];
        for (int32_t h = 0; h < hidden; ++h) {
            double a = (double)b1[h];
            const float *w = W1 + (int64_t)h * in;
            for (int32_t c = 0; c < in; ++c) a += (double)w[c] * e[c];
            if (a < 0.0) a = 0.0;
            o0 += (double)W2[h] * a;
            o1 += (double)W2[hidden + h] * a;
        }
        flow[2 * i] = o0;
        flow[2 * i + 1] = o1;
    }
    return ORC_OK;
}

/* Lemma 1: g_hat(q) = Re((1/D) sum_d emb[d] * conj(exp(i q . w_d))), with the query
 * offset q = (qt/dt, qx/dx, qy/dy) in the same normalised units as Eq. (emb). */
int oracle_kde_query(const double *emb, int32_t D, const double *T, const double *X,
                     const double *Y, double qt_over_dt, double qx_over_dx, double qy_over_dy,
                     double *out) {
    if (!emb || !T || !X || !Y || !out || D <= 0) return ORC_EINVAL;
    double s = 0.0;
    for (int32_t d = 0; d < D; ++d) {
        const double a = qt_over_dt * T[d] + qx_over_dx * X[d] + qy_over_dy * Y[d];
        s += emb[d] * cos(a) + emb[D + d] * sin(a);
    }
    *out = s / D;
    return ORC_OK;
}
