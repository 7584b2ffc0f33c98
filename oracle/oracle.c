/*
 * oracle.c -- plain, slow, FP64 CPU reference of the analytic Gaussian
 * line-integral projector and its adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * What it computes (paper section 3, "Method"):
 *   G(x)   = exp(-1/2 (x-mu)^T Sigma^-1 (x-mu)),  Sigma = R S S^T R^T   (Eq. 2)
 *   r(t)   = o + t d                                                   (Eq. 3)
 *   I(r)   = sum_i rho_i * int G_i(o + t d) dt                          (Eq. 4)
 *   delta  = o - mu,  A = d^T P d,  B = d^T P delta,  C = delta^T P delta,
 *            P = Sigma^-1                                               (Eq. 7)
 *   exponent along the ray = -1/2 (C + 2 B t + A t^2)                  (Eq. 8)
 *   over the whole line:  sqrt(2 pi / A) exp(-1/2 (C - B^2/A))          (Eqs. 9-11)
 *   I = sum_i rho_i sqrt(2 pi/A_i) exp(-1/2 (C_i - B_i^2/A_i))          (Eq. 12)
 * Finite segments [t_a, t_b] (not in the paper, which integrates over the
 * whole line): completing the square as in Eq. 9 and integrating the
 * Gaussian of Eq. 10 over a finite interval gives
 *   rho exp(-m/2) sqrt(pi/(2A)) [erf(w_b) - erf(w_a)],  w = (A t + B)/sqrt(2A),
 * which tends to Eq. 11 as t_a -> -inf, t_b -> +inf.
 *
 * "Skip Gaussians whose contributions are negligible" (section 4.1,
 * implementation details) is read as: a pair counts when m = C - B^2/A <= K^2
 * with K = 3, i.e. when the line meets the 3-sigma ellipsoid.  Pairs with
 * |m - K^2| <= band are ambiguous between FP32 and FP64 evaluation; they are
 * added to I_hi only, so I_lo <= I <= I_hi brackets every admissible result.
 *
 * Gradients (the paper only states the expression is differentiable): the
 * analytic derivative of each pair's contribution with respect to mu,
 * log-scale, the (unnormalised) quaternion and rho, chained through
 * Sigma^-1 = R(q/|q|) diag(exp(-2 l)) R^T.
 *
 * Geometries (section 3 "Inherent limitations" names cone/parallel-beam CT and
 * arc-corrected PET; their constants are this project's readings):
 *   kind 0  parallel-beam CT: e_w=(cos th, sin th, 0), e_u=(-sin th, cos th, 0),
 *           e_v=(0,0,1); o = u e_u + v e_v, d = e_w, t in [t_a, t_b].
 *   kind 1  cone-beam CT: same frame, source S = -dso e_w, detector point
 *           D = S + dsd e_w + u e_u + v e_v; o = S, d = (D-S)/|D-S|,
 *           t in [0, |D-S|].
 *   kind 2  PET ring: phi_j = pi j / n_views (or angles[j] when the caller
 *           gives the angles, e.g. a subset of a sinogram's angles),
 *           e_u=(cos phi, sin phi, 0),
 *           e_v=(0,0,1), e_w=(sin phi, -cos phi, 0); o = s e_u + z e_v,
 *           d = e_w, t in [-sqrt(R^2-s^2), +sqrt(R^2-s^2)].
 *           Arc-corrected: s_k = (k-c) pi R / n_crystals; raw chords:
 *           s_k = R sin((k-c) pi / n_crystals); c = (n_radial-1)/2.
 *   kind 3  fully 3-D PET: n_rows rings at z_r = (r - (n_rows-1)/2) pitch_v,
 *           the LORs between rings r1 and r2 = r1 + delta for every ring
 *           difference |delta| <= max_ring_diff, at the angles and radial
 *           bins of kind 2.  View v = (2 max_ring_diff + 1) segments x
 *           n_views angles: segment sg = v / n_views (delta = sg -
 *           max_ring_diff), angle a = v % n_views.  Row j is the ring pair
 *           r1 = j + max(0, -delta) (j < n_rows - |delta|; the other rows
 *           have no LOR and project to 0), at the mid-height
 *           z_mid = (z_r1 + z_r2)/2.  The LOR runs from
 *           s e_u - h e_w + z_r1 e_z to s e_u + h e_w + z_r2 e_z, h = sqrt(R^2 - s^2).
 *   Pixel coordinates: u_i = (i - (n_cols-1)/2) pitch_u, v_j likewise.
 *   Output layout: CT [view][row][col]; PET [plane][angle][radial];
 *   3-D PET [segment][angle][ring pair][radial].
 *   Time of flight (PET kinds, n_tof > 0): every LOR carries n_tof outputs,
 *   TOF bin k weighting the line by N(t; t_k, sigma_T^2) with t measured
 *   along the LOR from its midpoint and t_k = (k - (n_tof - 1)/2) spacing;
 *   output [k][the layout above].
 *
 * It also holds an FP32 replica of the culling predicate (records and
 * detector bounding boxes) used only to check that the GPU tile lists are
 * bit-exact; that replica is a specification written out in C, built with
 * -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t kind, n_views, n_rows, n_cols;
    const double *angles;
    double pitch_u, pitch_v, t_a, t_b, dso, dsd, radius;
    int32_t n_crystals, arc_mode, max_ring_diff;
    /* time of flight on PET LORs (n_tof = 0: none): n_tof bins centred at
     * t_k = (k - (n_tof - 1)/2) tof_spacing along the LOR from its midpoint,
     * each weighting the line by N(t; t_k, tof_sigma^2) */
    int32_t n_tof;
    double tof_spacing, tof_sigma;
} og_geom;

#define OG_PARALLEL 0
#define OG_CONE 1
#define OG_PET 2
#define OG_PET3D 3

/* number of views: 3-D PET has one per (segment, angle) */
static int og_nviews(const og_geom *g)
{
    return g->kind == OG_PET3D ? g->n_views * (2 * g->max_ring_diff + 1) : g->n_views;
}

/* outputs per LOR: its time-of-flight bins (1 without time of flight) */
static int og_tof_bins(const og_geom *g)
{
    return g->n_tof > 0 ? g->n_tof : 1;
}

/* centre (along the LOR from its midpoint) and 1/sigma^2 of TOF bin k (0, 0
 * without time of flight) */
static void og_tof(const og_geom *g, int k, double *tc, double *tau)
{
    *tc = 0.0;
    *tau = 0.0;
    if (g->n_tof > 0) {
        *tc = ((double)k - 0.5 * (double)(g->n_tof - 1)) * g->tof_spacing;
        *tau = 1.0 / (g->tof_sigma * g->tof_sigma);
    }
}

/* 3-D PET: ring difference of view v */
static int og_delta(const og_geom *g, int v)
{
    return v / g->n_views - g->max_ring_diff;
}

static const double OG_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* geometry (FP64)                                                     */
/* ------------------------------------------------------------------ */

static void og_frame(const og_geom *g, int v, double eu[3], double ev[3], double ew[3])
{
    if (g->kind == OG_PET || g->kind == OG_PET3D) {
        if (g->kind == OG_PET3D) v = v % g->n_views;
        double phi = g->angles ? g->angles[v] : (OG_PI * (double)v) / (double)g->n_views;
        double c = cos(phi), s = sin(phi);
        eu[0] = c;  eu[1] = s;  eu[2] = 0.0;
        ev[0] = 0.; ev[1] = 0.; ev[2] = 1.0;
        ew[0] = s;  ew[1] = -c; ew[2] = 0.0;
    } else {
        double th = g->angles[v];
        double c = cos(th), s = sin(th);
        ew[0] = c;  ew[1] = s;  ew[2] = 0.0;
        eu[0] = -s; eu[1] = c;  eu[2] = 0.0;
        ev[0] = 0.; ev[1] = 0.; ev[2] = 1.0;
    }
}

static double og_u(const og_geom *g, int i)
{
    double k = (double)i - 0.5 * (double)(g->n_cols - 1);
    if (g->kind == OG_PET || g->kind == OG_PET3D) {
        if (g->arc_mode == 0)
            return k * ((OG_PI * g->radius) / (double)g->n_crystals);
        return g->radius * sin((k * OG_PI) / (double)g->n_crystals);
    }
    return k * g->pitch_u;
}

static double og_v(const og_geom *g, int j)
{
    return ((double)j - 0.5 * (double)(g->n_rows - 1)) * g->pitch_v;
}

/* 3-D PET: mid-height of ring pair j in view v (its segment) */
static double og_v3(const og_geom *g, int v, int j)
{
    int ad = abs(og_delta(g, v));
    return ((double)j + 0.5 * (double)ad - 0.5 * (double)(g->n_rows - 1)) * g->pitch_v;
}

static int64_t og_index(const og_geom *g, int v, int j, int i)
{
    if (g->kind == OG_PET)
        return ((int64_t)j * g->n_views + v) * g->n_cols + i;
    return ((int64_t)v * g->n_rows + j) * g->n_cols + i;
}

/* the ray of pixel (v, j, i); returns 0 when the pixel has none (3-D PET rows
 * beyond the segment's ring pairs) */
static int og_ray(const og_geom *g, int v, int j, int i,
                  double o[3], double d[3], double *ta, double *tb)
{
    double eu[3], ev[3], ew[3];
    og_frame(g, v, eu, ev, ew);
    double u = og_u(g, i), w = og_v(g, j);
    if (g->kind == OG_PET3D) {
        int delta = og_delta(g, v);
        if (j >= g->n_rows - abs(delta)) {
            for (int k = 0; k < 3; k++) { o[k] = 0.0; d[k] = ew[k]; }
            *ta = *tb = 0.0;
            return 0;
        }
        double h = g->radius * g->radius - u * u;
        h = h > 0.0 ? sqrt(h) : 0.0;
        double zm = og_v3(g, v, j), dz = (double)delta * g->pitch_v;
        double L = sqrt(4.0 * h * h + dz * dz);
        for (int k = 0; k < 3; k++) {
            o[k] = u * eu[k] + zm * ev[k];
            d[k] = (2.0 * h * ew[k] + dz * ev[k]) / L;
        }
        *ta = -0.5 * L;
        *tb = 0.5 * L;
        return 1;
    }
    if (g->kind == OG_CONE) {
        double S[3], D[3], L = 0.0;
        for (int k = 0; k < 3; k++) {
            S[k] = -g->dso * ew[k];
            D[k] = S[k] + g->dsd * ew[k] + u * eu[k] + w * ev[k];
        }
        for (int k = 0; k < 3; k++) L += (D[k] - S[k]) * (D[k] - S[k]);
        L = sqrt(L);
        for (int k = 0; k < 3; k++) { o[k] = S[k]; d[k] = (D[k] - S[k]) / L; }
        *ta = 0.0;
        *tb = L;
    } else {
        for (int k = 0; k < 3; k++) { o[k] = u * eu[k] + w * ev[k]; d[k] = ew[k]; }
        if (g->kind == OG_PET) {
            double h = g->radius * g->radius - u * u;
            h = h > 0.0 ? sqrt(h) : 0.0;
            *ta = -h;
            *tb = h;
        } else {
            *ta = g->t_a;
            *tb = g->t_b;
        }
    }
    return 1;
}

static void og_unflatten(const og_geom *g, int64_t idx, int *v, int *j, int *i)
{
    *i = (int)(idx % g->n_cols);
    int64_t r = idx / g->n_cols;
    if (g->kind == OG_PET) { *v = (int)(r % g->n_views); *j = (int)(r / g->n_views); }
    else { *j = (int)(r % g->n_rows); *v = (int)(r / g->n_rows); }
}

/* ------------------------------------------------------------------ */
/* Gaussian parameters -> R, Sigma, P = Sigma^-1 (FP64), Eq. 2          */
/* ------------------------------------------------------------------ */

/* R(q/|q|) for q = (w, x, y, z); a zero quaternion is read as identity */
static void og_rot(const float *q, double R[3][3], double qn[4], double *qnorm)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double n = sqrt(w * w + x * x + y * y + z * z);
    if (!(n > 0.0)) { w = 1.0; x = y = z = 0.0; n = 1.0; }
    else { w /= n; x /= n; y /= n; z /= n; }
    qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z;
    *qnorm = n;
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

/* Sigma = R diag(e^{2l}) R^T and P = R diag(e^{-2l}) R^T */
static void og_cov(const float *ls, const float *q, double Sig[3][3], double P[3][3])
{
    double R[3][3], qn[4], qnorm;
    og_rot(q, R, qn, &qnorm);
    double s2[3], p2[3];
    for (int k = 0; k < 3; k++) { s2[k] = exp(2.0 * (double)ls[k]); p2[k] = exp(-2.0 * (double)ls[k]); }
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double s = 0.0, p = 0.0;
            for (int k = 0; k < 3; k++) { s += R[a][k] * R[b][k] * s2[k]; p += R[a][k] * R[b][k] * p2[k]; }
            Sig[a][b] = s;
            P[a][b] = p;
        }
}

/* ------------------------------------------------------------------ */
/* one Gaussian on one ray: Eqs. 7-11 (+ finite-segment erf)           */
/* ------------------------------------------------------------------ */

/* Phi = 1/2 [erf(wb) - erf(wa)], written with erfc where both ends share a sign */
static double og_phi(double wa, double wb)
{
    if (wa >= 0.0) return 0.5 * (erfc(wa) - erfc(wb));
    if (wb <= 0.0) return 0.5 * (erfc(-wb) - erfc(-wa));
    return 0.5 * (erf(wb) - erf(wa));
}

/*
 * Kernel of the primitives.  0: the Gaussian of Eq. 2.  1: the Epanechnikov
 * kernel named in section 2 as an alternative for ray tracing, read here as
 * rho (1 - m(x) / kappa^2)_+ with m(x) the Mahalanobis distance squared of
 * Eq. 2's covariance and kappa^2 = 7, so that the normalised kernel has
 * covariance Sigma (the Epanechnikov kernel on the unit 3-ball has variance
 * 1/7 per axis).  Selected by or_set_kernel for every following call.
 */
#define OG_KAPPA2 7.0
static int og_kern = 0;

void or_set_kernel(int kernel) { og_kern = kernel; }

typedef struct {
    double A, B, C, m, wa, wb, phi, K, f;  /* K = rho sqrt(2pi/A) e^{-m/2} */
    /* exponent of the value: m, or m' of the time-of-flight weighted form,
     * and the weight's normalisation factor (1 without time of flight) */
    double mv, sc;
    /* Epanechnikov: clipped interval [s0, s1] around the line's closest point
     * to mu (s = t + B/A); ea, eb: the ends are the segment's own */
    double s0, s1, c;
    int ea, eb;
} og_pairval;

/* Epanechnikov along the line: with c = 1 - m / kappa^2 the integrand is
 * rho (c - A s^2 / kappa^2) for |s| <= a = sqrt(kappa^2 c / A), so the
 * integral over [s0, s1] is rho [c s - A s^3 / (3 kappa^2)] between them */
static void og_eval_epan(double ta, double tb, double rho, og_pairval *r)
{
    r->c = 1.0 - r->m / OG_KAPPA2;
    r->s0 = r->s1 = 0.0;
    r->ea = r->eb = 0;
    r->K = 0.0;
    r->f = 0.0;
    if (!(r->m < OG_KAPPA2)) return;
    const double a = sqrt(OG_KAPPA2 * r->c / r->A);
    const double sa = ta + r->B / r->A, sb = tb + r->B / r->A;
    r->ea = sa > -a;
    r->eb = sb < a;
    r->s0 = r->ea ? sa : -a;
    r->s1 = r->eb ? sb : a;
    if (!(r->s1 > r->s0)) { r->s0 = r->s1 = 0.0; r->ea = r->eb = 0; return; }
    const double F1 = r->c * r->s1 - r->A * r->s1 * r->s1 * r->s1 / (3.0 * OG_KAPPA2);
    const double F0 = r->c * r->s0 - r->A * r->s0 * r->s0 * r->s0 / (3.0 * OG_KAPPA2);
    r->K = F1 - F0;            /* value per unit rho */
    r->f = rho * r->K;
}

/*
 * Time of flight (the paper's future-work section plans TOF PET): a ray may
 * carry a Gaussian weight N(t; t_c, sigma_T^2) along itself (tau = 1 /
 * sigma_T^2; tau = 0: none).  The weighted integrand exp(-(A t^2 + 2 B t +
 * C)/2) N(t) is again of the form of Eq. 7 with A' = A + tau, B' = B - tau t_c,
 * C' = C + tau t_c^2 and the factor sqrt(tau / 2 pi); the pair still counts by
 * its spatial m (the 3-sigma cut).
 */
static void og_eval(const double o[3], const double d[3], double ta, double tb,
                    const double mu[3], double P[3][3], double rho, double tc, double tau,
                    og_pairval *r)
{
    double del[3] = { o[0] - mu[0], o[1] - mu[1], o[2] - mu[2] };
    double Pd[3], Pdel[3];
    for (int a = 0; a < 3; a++) {
        Pd[a] = P[a][0] * d[0] + P[a][1] * d[1] + P[a][2] * d[2];
        Pdel[a] = P[a][0] * del[0] + P[a][1] * del[1] + P[a][2] * del[2];
    }
    r->A = d[0] * Pd[0] + d[1] * Pd[1] + d[2] * Pd[2];            /* Eq. 7 */
    r->B = d[0] * Pdel[0] + d[1] * Pdel[1] + d[2] * Pdel[2];
    r->C = del[0] * Pdel[0] + del[1] * Pdel[1] + del[2] * Pdel[2];
    r->m = r->C - r->B * r->B / r->A;                              /* Eq. 9 */
    r->mv = r->m;
    r->sc = 1.0;
    if (og_kern == 1) {
        og_eval_epan(ta, tb, rho, r);
        return;
    }
    double scale = 1.0;
    if (tau > 0.0) {
        r->A += tau;
        r->B -= tau * tc;
        r->C += tau * tc * tc;
        r->mv = r->C - r->B * r->B / r->A;
        scale = sqrt(tau / (2.0 * OG_PI));
        r->sc = scale;
    }
    double s2A = sqrt(2.0 * r->A);
    r->wa = (r->A * ta + r->B) / s2A;
    r->wb = (r->A * tb + r->B) / s2A;
    r->phi = og_phi(r->wa, r->wb);
    r->K = scale * rho * sqrt(2.0 * OG_PI / r->A) * exp(-0.5 * r->mv);      /* Eq. 11 */
    r->f = r->K * r->phi;
}

/* derivatives of one pair's contribution w.r.t. mu (3), P (full symmetric
 * matrix gradient, 3x3) and rho; returns through gm, gP, grho (added, scaled by w) */
static void og_pair_grad(const double o[3], const double d[3], double ta, double tb,
                         const double mu[3], double P[3][3], double rho, double wgt,
                         const og_pairval *r, double gm[3], double gP[3][3], double *grho)
{
    const double A = r->A, B = r->B;
    double del[3] = { o[0] - mu[0], o[1] - mu[1], o[2] - mu[2] };
    if (og_kern == 1) {
        /* Leibniz: the clipped ends at +-a carry a zero integrand; the
         * segment's own ends move with B and A through s = t + B/A */
        if (!(r->s1 > r->s0)) return;
        const double L = r->s1 - r->s0, k2 = OG_KAPPA2;
        const double phi1 = r->eb ? rho * (r->c - A * r->s1 * r->s1 / k2) : 0.0;
        const double phi0 = r->ea ? rho * (r->c - A * r->s0 * r->s0 / k2) : 0.0;
        const double fC = -rho * L / k2;
        const double fB = rho * (2.0 * B / A) * L / k2 + (phi1 - phi0) / A;
        const double fA = -rho * ((B * B) / (A * A) * L
                                  + (r->s1 * r->s1 * r->s1 - r->s0 * r->s0 * r->s0) / 3.0) / k2
                          - (phi1 - phi0) * B / (A * A);
        double Pd[3], Pdel[3];
        for (int a = 0; a < 3; a++) {
            Pd[a] = P[a][0] * d[0] + P[a][1] * d[1] + P[a][2] * d[2];
            Pdel[a] = P[a][0] * del[0] + P[a][1] * del[1] + P[a][2] * del[2];
        }
        for (int a = 0; a < 3; a++) gm[a] += wgt * (-fB * Pd[a] - 2.0 * fC * Pdel[a]);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                gP[a][b] += wgt * (fA * d[a] * d[b] + fB * 0.5 * (d[a] * del[b] + del[a] * d[b])
                                   + fC * del[a] * del[b]);
        *grho += wgt * r->K;
        return;
    }
    double ea = exp(-r->wa * r->wa), eb = exp(-r->wb * r->wb);
    if (!isfinite(r->wa)) ea = 0.0;
    if (!isfinite(r->wb)) eb = 0.0;
    double eta = isfinite(ta) ? ta : 0.0, etb = isfinite(tb) ? tb : 0.0;
    double dPhi_dB = (eb - ea) / sqrt(2.0 * OG_PI * A);
    double dPhi_dA = (eb * (A * etb - B) - ea * (A * eta - B)) / (sqrt(OG_PI) * pow(2.0 * A, 1.5));
    double fC = -0.5 * r->f;
    double fB = r->f * B / A + r->K * dPhi_dB;
    double fA = -0.5 * r->f / A - 0.5 * r->f * B * B / (A * A) + r->K * dPhi_dA;
    double Pd[3], Pdel[3];
    for (int a = 0; a < 3; a++) {
        Pd[a] = P[a][0] * d[0] + P[a][1] * d[1] + P[a][2] * d[2];
        Pdel[a] = P[a][0] * del[0] + P[a][1] * del[1] + P[a][2] * del[2];
    }
    /* dB/dmu = -P d, dC/dmu = -2 P delta */
    for (int a = 0; a < 3; a++) gm[a] += wgt * (-fB * Pd[a] - 2.0 * fC * Pdel[a]);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            gP[a][b] += wgt * (fA * d[a] * d[b] + fB * 0.5 * (d[a] * del[b] + del[a] * d[b])
                               + fC * del[a] * del[b]);
    *grho += wgt * (rho != 0.0 ? r->f / rho
                               : r->sc * sqrt(2.0 * OG_PI / A) * exp(-0.5 * r->mv) * r->phi);
}

/* dL/dP (symmetric) and the parameters -> dL/dl, dL/dq  (P = R diag(e^{-2l}) R^T) */
static void og_chain(const float *ls, const float *q, double gP[3][3], double gl[3], double gq[4])
{
    double R[3][3], qn[4], qnorm;
    og_rot(q, R, qn, &qnorm);
    double D[3];
    for (int k = 0; k < 3; k++) D[k] = exp(-2.0 * (double)ls[k]);
    double G[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) G[a][b] = 0.5 * (gP[a][b] + gP[b][a]);
    /* dL/dD_k = r_k^T G r_k,  dD_k/dl_k = -2 D_k */
    for (int k = 0; k < 3; k++) {
        double s = 0.0;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) s += R[a][k] * G[a][b] * R[b][k];
        gl[k] = -2.0 * D[k] * s;
    }
    /* dL/dR = 2 G R D */
    double gR[3][3];
    for (int a = 0; a < 3; a++)
        for (int k = 0; k < 3; k++) {
            double s = 0.0;
            for (int b = 0; b < 3; b++) s += G[a][b] * R[b][k];
            gR[a][k] = 2.0 * s * D[k];
        }
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    /* dR_ab / d(w,x,y,z) for the unit-quaternion rotation matrix */
    double dR[4][3][3] = {
        { { 0, -2 * z, 2 * y }, { 2 * z, 0, -2 * x }, { -2 * y, 2 * x, 0 } },
        { { 0, 2 * y, 2 * z }, { 2 * y, -4 * x, -2 * w }, { 2 * z, 2 * w, -4 * x } },
        { { -4 * y, 2 * x, 2 * w }, { 2 * x, 0, 2 * z }, { -2 * w, 2 * z, -4 * y } },
        { { -4 * z, -2 * w, 2 * x }, { 2 * w, -4 * z, 2 * y }, { 2 * x, 2 * y, 0 } },
    };
    double gqn[4];
    for (int c = 0; c < 4; c++) {
        double s = 0.0;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) s += gR[a][b] * dR[c][a][b];
        gqn[c] = s;
    }
    /* qn = q/|q|  =>  dL/dq = (gqn - qn (qn . gqn)) / |q| */
    double dot = gqn[0] * qn[0] + gqn[1] * qn[1] + gqn[2] * qn[2] + gqn[3] * qn[3];
    for (int c = 0; c < 4; c++) gq[c] = (gqn[c] - qn[c] * dot) / qnorm;
}

/* ------------------------------------------------------------------ */
/* per-(Gaussian, view) detector bounding box in FP64 (oracle's own)   */
/* ------------------------------------------------------------------ */

static int og_lower(const double *tab, int n, double x)   /* first i with tab[i] >= x */
{
    int lo = 0, hi = n;
    while (lo < hi) { int mid = (lo + hi) >> 1; if (tab[mid] >= x) hi = mid; else lo = mid + 1; }
    return lo;
}
static int og_upper(const double *tab, int n, double x)   /* last i with tab[i] <= x */
{
    int lo = 0, hi = n;
    while (lo < hi) { int mid = (lo + hi) >> 1; if (tab[mid] > x) hi = mid; else lo = mid + 1; }
    return lo - 1;
}

static double og_quad(double Sig[3][3], const double a[3], const double b[3])
{
    double s = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) s += a[i] * Sig[i][j] * b[j];
    return s;
}

/* interval of detector coordinate along axis e (u or v) whose rays meet the
 * K-sigma ellipsoid (exact tangent planes); returns 0 if unbounded */
static int og_cone_interval(double K2, double dsd, double a_e, double a_w,
                            double s_ee, double s_ew, double s_ww, double *lo, double *hi)
{
    double alpha = a_w * a_w - K2 * s_ww;
    if (!(alpha > 0.0)) return 0;
    double beta = dsd * (a_e * a_w - K2 * s_ew);
    double disc = a_w * a_w * s_ee - 2.0 * a_e * a_w * s_ew + a_e * a_e * s_ww - K2 * (s_ee * s_ww - s_ew * s_ew);
    if (disc < 0.0) disc = 0.0;
    double r = dsd * sqrt(K2 * disc);
    *lo = (beta - r) / alpha;
    *hi = (beta + r) / alpha;
    return 1;
}

static void og_bbox(const og_geom *g, int v, const double mu[3], double Sig[3][3], double K2,
                    const double *utab, const double *vtab, int *i0, int *i1, int *j0, int *j1)
{
    double eu[3], ev[3], ew[3];
    og_frame(g, v, eu, ev, ew);
    double mu_u = mu[0] * eu[0] + mu[1] * eu[1] + mu[2] * eu[2];
    double mu_v = mu[0] * ev[0] + mu[1] * ev[1] + mu[2] * ev[2];
    double ulo = -INFINITY, uhi = INFINITY, vlo = -INFINITY, vhi = INFINITY;
    if (g->kind == OG_CONE) {
        double mu_w = mu[0] * ew[0] + mu[1] * ew[1] + mu[2] * ew[2];
        double a_w = mu_w + g->dso;
        double suu = og_quad(Sig, eu, eu), svv = og_quad(Sig, ev, ev), sww = og_quad(Sig, ew, ew);
        double suw = og_quad(Sig, eu, ew), svw = og_quad(Sig, ev, ew);
        double lo, hi;
        if (og_cone_interval(K2, g->dsd, mu_u, a_w, suu, suw, sww, &lo, &hi)) { ulo = lo; uhi = hi; }
        if (og_cone_interval(K2, g->dsd, mu_v, a_w, svv, svw, sww, &lo, &hi)) { vlo = lo; vhi = hi; }
    } else {
        double hu = sqrt(K2 * og_quad(Sig, eu, eu)), hv = sqrt(K2 * og_quad(Sig, ev, ev));
        ulo = mu_u - hu; uhi = mu_u + hu; vlo = mu_v - hv; vhi = mu_v + hv;
    }
    *i0 = og_lower(utab, g->n_cols, ulo);
    *i1 = og_upper(utab, g->n_cols, uhi);
    if (g->kind == OG_PET3D) {
        /* the LOR at (s, z_mid) has z = z_mid + slope w (w along e_w), slope =
         * dz / (2 h(s)): it meets the ellipsoid only if z_mid lies in
         * mu_z - slope mu_w +- sqrt(K2 a^T Sigma a), a = e_z - slope e_w; over
         * the box's s-range the slope spans [dz/2h_max, dz/2h_min] and the
         * union of those intervals is bounded by its end slopes */
        int delta = og_delta(g, v), ad = abs(delta);
        double dz = (double)delta * g->pitch_v;
        double mu_w = mu[0] * ew[0] + mu[1] * ew[1] + mu[2] * ew[2];
        double slo_ = ulo < utab[0] ? utab[0] : ulo, shi_ = uhi > utab[g->n_cols - 1] ? utab[g->n_cols - 1] : uhi;
        double amin = (slo_ <= 0.0 && shi_ >= 0.0) ? 0.0 : fmin(fabs(slo_), fabs(shi_));
        double amax = fmax(fabs(slo_), fabs(shi_));
        double R2 = g->radius * g->radius;
        double hmax = sqrt(fmax(R2 - amin * amin, 0.0)), hmin = sqrt(fmax(R2 - amax * amax, 0.0));
        int last = g->n_rows - ad - 1;
        if (!(hmin > 0.0)) {            /* the box reaches the ring's edge: slopes unbounded */
            *j0 = 0;
            *j1 = last;
            return;
        }
        double zl = INFINITY, zh = -INFINITY;
        for (int e = 0; e < 2; e++) {
            double hh = e ? hmin : hmax;
            double sl = dz / (2.0 * hh);
            double a[3] = { -sl * ew[0], -sl * ew[1], 1.0 - sl * ew[2] };
            double c = mu[2] - sl * mu_w, half = sqrt(K2 * og_quad(Sig, a, a));
            zl = fmin(zl, c - half);
            zh = fmax(zh, c + half);
        }
        double off = 0.5 * (double)ad - 0.5 * (double)(g->n_rows - 1);
        double jl = ceil(zl / g->pitch_v - off), jh = floor(zh / g->pitch_v - off);
        *j0 = jl < 0.0 ? 0 : (jl > last + 1 ? last + 1 : (int)jl);
        *j1 = jh > last ? last : (jh < -1.0 ? -1 : (int)jh);
        return;
    }
    *j0 = og_lower(vtab, g->n_rows, vlo);
    *j1 = og_upper(vtab, g->n_rows, vhi);
}

/* bounding-box factor for the oracle's own loop: 3.05 sigma for the 3-sigma
 * cut, scaled with the cut (a cut at +inf visits the whole detector) */
static double og_box_k2(double cut2, double band)
{
    return (cut2 + band) * ((3.05 * 3.05) / 9.0);
}

static void og_tables(const og_geom *g, double **ut, double **vt)
{
    *ut = (double *)malloc(sizeof(double) * (size_t)(g->n_cols > 0 ? g->n_cols : 1));
    *vt = (double *)malloc(sizeof(double) * (size_t)(g->n_rows > 0 ? g->n_rows : 1));
    for (int i = 0; i < g->n_cols; i++) (*ut)[i] = og_u(g, i);
    for (int j = 0; j < g->n_rows; j++) (*vt)[j] = og_v(g, j);
}

static void og_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* ------------------------------------------------------------------ */
/* exported API                                                         */
/* ------------------------------------------------------------------ */

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* single pair: out = {value, m, A, B, C} (no cut-off applied) */
void or_pair(const double *o, const double *d, double ta, double tb,
             const float *mu, const float *ls, const float *q, float rho, double *out)
{
    double Sig[3][3], P[3][3], m3[3] = { mu[0], mu[1], mu[2] };
    og_cov(ls, q, Sig, P);
    og_pairval r;
    og_eval(o, d, ta, tb, m3, P, rho, 0.0, 0.0, &r);
    out[0] = r.f; out[1] = r.m; out[2] = r.A; out[3] = r.B; out[4] = r.C;
}

/* single pair gradient: out = d value / d(mu[3], l[3], q[4], rho) */
void or_pair_grad(const double *o, const double *d, double ta, double tb,
                  const float *mu, const float *ls, const float *q, float rho, double *out)
{
    double Sig[3][3], P[3][3], m3[3] = { mu[0], mu[1], mu[2] };
    og_cov(ls, q, Sig, P);
    og_pairval r;
    og_eval(o, d, ta, tb, m3, P, rho, 0.0, 0.0, &r);
    double gm[3] = { 0, 0, 0 }, gP[3][3] = { { 0 } }, grho = 0.0, gl[3], gq[4];
    og_pair_grad(o, d, ta, tb, m3, P, rho, 1.0, &r, gm, gP, &grho);
    og_chain(ls, q, gP, gl, gq);
    for (int k = 0; k < 3; k++) { out[k] = gm[k]; out[3 + k] = gl[k]; }
    for (int k = 0; k < 4; k++) out[6 + k] = gq[k];
    out[10] = grho;
}

/* full matrices Sigma and P for n Gaussians (row-major 3x3 each) */
void or_cov(int64_t n, const float *ls, const float *q, double *sig9, double *p9)
{
    for (int64_t g = 0; g < n; g++) {
        double S[3][3], P[3][3];
        og_cov(ls + 3 * g, q + 4 * g, S, P);
        memcpy(sig9 + 9 * g, S, sizeof(S));
        memcpy(p9 + 9 * g, P, sizeof(P));
    }
}

/* LORs / detector rays of the geometry (one per pixel of every view) */
static int64_t og_num_lors(const og_geom *g)
{
    return (int64_t)og_nviews(g) * g->n_rows * g->n_cols;
}

/* outputs: with time of flight, TOF bin k of LOR x is output k * lors + x */
int64_t or_num_rays(const og_geom *g)
{
    return og_num_lors(g) * og_tof_bins(g);
}

/* rays for flat output indices (the LOR of a time-of-flight output) */
void or_rays(const og_geom *g, int64_t n, const int64_t *idx, double *o, double *d, double *ta, double *tb)
{
    const int64_t nl = og_num_lors(g);
    for (int64_t r = 0; r < n; r++) {
        int v, j, i;
        og_unflatten(g, idx[r] % nl, &v, &j, &i);
        og_ray(g, v, j, i, o + 3 * r, d + 3 * r, ta + r, tb + r);
    }
}

/* pixel coordinate tables (u per column, v per row) as the oracle defines them */
void or_tables(const og_geom *g, double *u, double *v)
{
    for (int i = 0; i < g->n_cols; i++) u[i] = og_u(g, i);
    for (int j = 0; j < g->n_rows; j++) v[j] = og_v(g, j);
}

static void og_accum(double f, double m, double cut2, double band, double *I, double *Ilo, double *Ihi)
{
    if (m <= cut2 - band) { *I += f; *Ilo += f; *Ihi += f; }
    else if (m <= cut2 + band) { if (m <= cut2) *I += f; *Ihi += f; }
}

/*
 * forward projection of every ray of the geometry.  brute != 0 evaluates
 * every (ray, Gaussian) pair; otherwise each (Gaussian, view) visits only the
 * pixels of its FP64 detector box (3.05 sigma), which contains all pairs
 * with m <= cut2 + band.  Sums run in Gaussian order per pixel.
 */
void or_forward(const og_geom *g, int64_t n, const float *mu, const float *ls, const float *q,
                const float *rho, double cut2, double band, int brute, int nthreads,
                double *I, double *Ilo, double *Ihi, int64_t *pairs)
{
    og_set_threads(nthreads);
    int64_t R = or_num_rays(g);
    memset(I, 0, sizeof(double) * (size_t)R);
    memset(Ilo, 0, sizeof(double) * (size_t)R);
    memset(Ihi, 0, sizeof(double) * (size_t)R);
    double *ut, *vt;
    og_tables(g, &ut, &vt);
    double (*Sig)[3][3] = malloc(sizeof(double[3][3]) * (size_t)(n > 0 ? n : 1));
    double (*P)[3][3] = malloc(sizeof(double[3][3]) * (size_t)(n > 0 ? n : 1));
    for (int64_t k = 0; k < n; k++) og_cov(ls + 3 * k, q + 4 * k, Sig[k], P[k]);
    int64_t npair = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : npair)
    for (int v = 0; v < og_nviews(g); v++) {
        for (int64_t k = 0; k < n; k++) {
            double m3[3] = { mu[3 * k], mu[3 * k + 1], mu[3 * k + 2] };
            int i0 = 0, i1 = g->n_cols - 1, j0 = 0, j1 = g->n_rows - 1;
            if (!brute) og_bbox(g, v, m3, Sig[k], og_box_k2(cut2, band), ut, vt, &i0, &i1, &j0, &j1);
            for (int j = j0; j <= j1; j++)
                for (int i = i0; i <= i1; i++) {
                    double o[3], d[3], ta, tb;
                    if (!og_ray(g, v, j, i, o, d, &ta, &tb)) continue;
                    for (int b = 0; b < og_tof_bins(g); b++) {
                        double tc, tau;
                        og_tof(g, b, &tc, &tau);
                        og_pairval r;
                        og_eval(o, d, ta, tb, m3, P[k], rho[k], tc, tau, &r);
                        int64_t x = og_index(g, v, j, i) + b * og_num_lors(g);
                        og_accum(r.f, r.m, cut2, band, I + x, Ilo + x, Ihi + x);
                        if (b == 0 && r.m <= cut2) npair++;
                    }
                }
        }
    }
    if (pairs) *pairs = npair;
    free(Sig); free(P); free(ut); free(vt);
}

/* brute-force forward projection of selected rays (flat indices) */
void or_forward_rays(const og_geom *g, int64_t n, const float *mu, const float *ls, const float *q,
                     const float *rho, double cut2, double band, int64_t nr, const int64_t *idx,
                     int nthreads, double *I, double *Ilo, double *Ihi)
{
    og_set_threads(nthreads);
    double (*P)[3][3] = malloc(sizeof(double[3][3]) * (size_t)(n > 0 ? n : 1));
    for (int64_t k = 0; k < n; k++) { double S[3][3]; og_cov(ls + 3 * k, q + 4 * k, S, P[k]); }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nr; r++) {
        int v, j, i;
        og_unflatten(g, idx[r] % og_num_lors(g), &v, &j, &i);
        double tc, tau;
        og_tof(g, (int)(idx[r] / og_num_lors(g)), &tc, &tau);
        double o[3], d[3], ta, tb;
        const int has = og_ray(g, v, j, i, o, d, &ta, &tb);
        double s = 0.0, slo = 0.0, shi = 0.0;
        if (!has) { I[r] = Ilo[r] = Ihi[r] = 0.0; continue; }
        for (int64_t k = 0; k < n; k++) {
            double m3[3] = { mu[3 * k], mu[3 * k + 1], mu[3 * k + 2] };
            og_pairval pv;
            og_eval(o, d, ta, tb, m3, P[k], rho[k], tc, tau, &pv);
            og_accum(pv.f, pv.m, cut2, band, &s, &slo, &shi);
        }
        I[r] = s; Ilo[r] = slo; Ihi[r] = shi;
    }
    free(P);
}

/* one Gaussian's gradient sums: unambiguous pairs (gm, gP, grho, chained at
 * the end) and, per parameter, the nominal / negative / positive sums of the
 * pairs within the band of the cut (each chained on its own) */
typedef struct {
    double gm[3], gP[3][3], grho;
    double bnom[11], bneg[11], bpos[11];
} og_gradacc;

static void og_grad_pair(og_gradacc *a, const double o[3], const double d[3], double ta, double tb,
                         double tc, double tau, const double m3[3], double P[3][3], double rho,
                         double w, double cut2, double band, const float *ls, const float *q)
{
    og_pairval r;
    og_eval(o, d, ta, tb, m3, P, rho, tc, tau, &r);
    if (!(r.m <= cut2 + band) || w == 0.0) return;
    if (r.m <= cut2 - band) {
        og_pair_grad(o, d, ta, tb, m3, P, rho, w, &r, a->gm, a->gP, &a->grho);
        return;
    }
    /* ambiguous pair: its own full parameter gradient */
    double bm[3] = { 0, 0, 0 }, bP[3][3] = { { 0 } }, br = 0.0, bl[3], bq[4], b[11];
    og_pair_grad(o, d, ta, tb, m3, P, rho, w, &r, bm, bP, &br);
    og_chain(ls, q, bP, bl, bq);
    for (int c = 0; c < 3; c++) { b[c] = bm[c]; b[3 + c] = bl[c]; }
    for (int c = 0; c < 4; c++) b[6 + c] = bq[c];
    b[10] = br;
    for (int c = 0; c < 11; c++) {
        if (r.m <= cut2) a->bnom[c] += b[c];
        if (b[c] < 0) a->bneg[c] += b[c]; else a->bpos[c] += b[c];
    }
}

static void og_grad_finish(og_gradacc *a, int64_t k, const float *ls, const float *q, double *g_mu,
                           double *g_ls, double *g_q, double *g_rho, double *lohi)
{
    double gl[3], gq[4], mainv[11];
    og_chain(ls, q, a->gP, gl, gq);
    for (int c = 0; c < 3; c++) { mainv[c] = a->gm[c]; mainv[3 + c] = gl[c]; }
    for (int c = 0; c < 4; c++) mainv[6 + c] = gq[c];
    mainv[10] = a->grho;
    for (int c = 0; c < 3; c++) {
        g_mu[3 * k + c] = mainv[c] + a->bnom[c];
        g_ls[3 * k + c] = mainv[3 + c] + a->bnom[3 + c];
    }
    for (int c = 0; c < 4; c++) g_q[4 * k + c] = mainv[6 + c] + a->bnom[6 + c];
    g_rho[k] = mainv[10] + a->bnom[10];
    if (lohi)
        for (int c = 0; c < 11; c++) {
            lohi[22 * k + c] = mainv[c] + a->bneg[c];
            lohi[22 * k + 11 + c] = mainv[c] + a->bpos[c];
        }
}

/*
 * adjoint: dL/d(mu, l, q, rho) = sum over pairs with m <= cut2 of
 * dLdI[ray] * d(contribution)/d(parameter).  sel (length nsel) restricts the
 * Gaussians evaluated (others are left untouched); sel == NULL means all.
 * Pairs with |m - cut2| <= band may be kept or dropped by an FP32
 * evaluation; when lohi != NULL it receives, per Gaussian, the bounds
 * lo[11] = main + sum of the negative parts of the band pairs' gradients and
 * hi[11] = main + sum of their positive parts (order mu[3], l[3], q[4], rho),
 * which bracket every admissible choice.
 */
void or_backward(const og_geom *g, int64_t n, const float *mu, const float *ls, const float *q,
                 const float *rho, double cut2, double band, const double *dLdI, int64_t nsel,
                 const int64_t *sel, int brute, int nthreads, double *g_mu, double *g_ls,
                 double *g_q, double *g_rho, double *lohi)
{
    og_set_threads(nthreads);
    double *ut, *vt;
    og_tables(g, &ut, &vt);
    int64_t cnt = sel ? nsel : n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < cnt; s++) {
        int64_t k = sel ? sel[s] : s;
        double Sig[3][3], P[3][3];
        og_cov(ls + 3 * k, q + 4 * k, Sig, P);
        double m3[3] = { mu[3 * k], mu[3 * k + 1], mu[3 * k + 2] };
        og_gradacc acc;
        memset(&acc, 0, sizeof(acc));
        for (int v = 0; v < og_nviews(g); v++) {
            int i0 = 0, i1 = g->n_cols - 1, j0 = 0, j1 = g->n_rows - 1;
            if (!brute) og_bbox(g, v, m3, Sig, og_box_k2(cut2, band), ut, vt, &i0, &i1, &j0, &j1);
            for (int j = j0; j <= j1; j++)
                for (int i = i0; i <= i1; i++) {
                    double o[3], d[3], ta, tb;
                    if (!og_ray(g, v, j, i, o, d, &ta, &tb)) continue;
                    for (int b = 0; b < og_tof_bins(g); b++) {
                        double tc, tau;
                        og_tof(g, b, &tc, &tau);
                        og_grad_pair(&acc, o, d, ta, tb, tc, tau, m3, P, rho[k],
                                     dLdI[og_index(g, v, j, i) + b * og_num_lors(g)], cut2, band, ls + 3 * k,
                                     q + 4 * k);
                    }
                }
        }
        og_grad_finish(&acc, k, ls + 3 * k, q + 4 * k, g_mu, g_ls, g_q, g_rho, lohi);
    }
    free(ut); free(vt);
}

/*
 * Explicit rays (any set of lines): ray r runs through o[3r..3r+2] along
 * d[3r..3r+2] (any nonzero length; normalised here), over t in
 * [t[2r], t[2r+1]] measured along the unit direction (+-inf allowed).
 * Every (ray, Gaussian) pair is evaluated: the plain definition, Eqs. 7-12
 * with the cut m <= cut2 and the band bracket as above.  tof (may be null):
 * per ray the time-of-flight centre and width (Gaussian kernel only).
 */
static void og_list_ray(const double *o, const double *d, const double *t, const double *tof, int64_t r,
                        double oo[3], double dd[3], double *ta, double *tb, double *tc, double *tau)
{
    double len = sqrt(d[3 * r] * d[3 * r] + d[3 * r + 1] * d[3 * r + 1] + d[3 * r + 2] * d[3 * r + 2]);
    for (int c = 0; c < 3; c++) { oo[c] = o[3 * r + c]; dd[c] = d[3 * r + c] / len; }
    *ta = t[2 * r];
    *tb = t[2 * r + 1];
    /* time of flight: tof[2r] = centre t_c, tof[2r + 1] = sigma_T (<= 0 or inf: none) */
    *tc = 0.0;
    *tau = 0.0;
    if (tof && tof[2 * r + 1] > 0.0 && isfinite(tof[2 * r + 1])) {
        *tc = tof[2 * r];
        *tau = 1.0 / (tof[2 * r + 1] * tof[2 * r + 1]);
    }
}

void or_forward_list(int64_t nr, const double *o, const double *d, const double *t, const double *tof,
                     int64_t n,
                     const float *mu, const float *ls, const float *q, const float *rho, double cut2,
                     double band, int nthreads, double *I, double *Ilo, double *Ihi, int64_t *pairs)
{
    og_set_threads(nthreads);
    double (*P)[3][3] = malloc(sizeof(double[3][3]) * (size_t)(n > 0 ? n : 1));
    for (int64_t k = 0; k < n; k++) { double S[3][3]; og_cov(ls + 3 * k, q + 4 * k, S, P[k]); }
    int64_t npair = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : npair)
    for (int64_t r = 0; r < nr; r++) {
        double oo[3], dd[3], ta, tb, tc, tau, s = 0.0, slo = 0.0, shi = 0.0;
        og_list_ray(o, d, t, tof, r, oo, dd, &ta, &tb, &tc, &tau);
        for (int64_t k = 0; k < n; k++) {
            double m3[3] = { mu[3 * k], mu[3 * k + 1], mu[3 * k + 2] };
            og_pairval pv;
            og_eval(oo, dd, ta, tb, m3, P[k], rho[k], tc, tau, &pv);
            og_accum(pv.f, pv.m, cut2, band, &s, &slo, &shi);
            if (pv.m <= cut2) npair++;
        }
        I[r] = s; Ilo[r] = slo; Ihi[r] = shi;
    }
    if (pairs) *pairs = npair;
    free(P);
}

void or_backward_list(int64_t nr, const double *o, const double *d, const double *t, const double *tof,
                      int64_t n,
                      const float *mu, const float *ls, const float *q, const float *rho, double cut2,
                      double band, const double *dLdI, int nthreads, double *g_mu, double *g_ls,
                      double *g_q, double *g_rho, double *lohi)
{
    og_set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n; k++) {
        double Sig[3][3], P[3][3];
        og_cov(ls + 3 * k, q + 4 * k, Sig, P);
        double m3[3] = { mu[3 * k], mu[3 * k + 1], mu[3 * k + 2] };
        og_gradacc acc;
        memset(&acc, 0, sizeof(acc));
        for (int64_t r = 0; r < nr; r++) {
            double oo[3], dd[3], ta, tb, tc, tau;
            og_list_ray(o, d, t, tof, r, oo, dd, &ta, &tb, &tc, &tau);
            og_grad_pair(&acc, oo, dd, ta, tb, tc, tau, m3, P, rho[k], dLdI[r], cut2, band, ls + 3 * k,
                         q + 4 * k);
        }
        og_grad_finish(&acc, k, ls + 3 * k, q + 4 * k, g_mu, g_ls, g_q, g_rho, lohi);
    }
}

/*
 * Voxelisation: the density field of the Gaussians (the integrand of Eq. 4,
 * rho exp(-1/2 (x - mu)^T P (x - mu)), Eq. 2) sampled at voxel centres
 * x = origin + (i, j, k) * size, with the same cut as the projector: a
 * Gaussian counts at x when its Mahalanobis distance squared is <= cut2
 * (band bracket as for projections).  Output layout [k][j][i]; sums run in
 * Gaussian order per voxel.  Each Gaussian visits the voxels of its FP64 box
 * of radius sqrt((cut2 + band) Sigma_aa) per axis, which holds every voxel
 * where it counts (or all voxels when brute != 0).
 */
void or_voxelize(const double *origin, const double *size, const int32_t *dims, int64_t n,
                 const float *mu, const float *ls, const float *q, const float *rho, double cut2,
                 double band, int brute, int nthreads, double *V, double *Vlo, double *Vhi)
{
    og_set_threads(nthreads);
    const int nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t nvox = (int64_t)nx * ny * nz;
    memset(V, 0, sizeof(double) * (size_t)nvox);
    memset(Vlo, 0, sizeof(double) * (size_t)nvox);
    memset(Vhi, 0, sizeof(double) * (size_t)nvox);
    double (*Sig)[3][3] = malloc(sizeof(double[3][3]) * (size_t)(n > 0 ? n : 1));
    double (*P)[3][3] = malloc(sizeof(double[3][3]) * (size_t)(n > 0 ? n : 1));
    for (int64_t k = 0; k < n; k++) og_cov(ls + 3 * k, q + 4 * k, Sig[k], P[k]);
    /* parallel over z slices: every voxel is written by one thread, Gaussians in order */
#pragma omp parallel for schedule(dynamic, 1)
    for (int kz = 0; kz < nz; kz++) {
        const double z = origin[2] + kz * size[2];
        for (int64_t g = 0; g < n; g++) {
            const double m3[3] = { mu[3 * g], mu[3 * g + 1], mu[3 * g + 2] };
            int lo[2] = { 0, 0 }, hi[2] = { nx - 1, ny - 1 };
            if (!brute) {
                const double r2 = cut2 + band;
                const double hz = sqrt(r2 * Sig[g][2][2]);
                if (z < m3[2] - hz || z > m3[2] + hz) continue;
                for (int a = 0; a < 2; a++) {
                    const double h = sqrt(r2 * Sig[g][a][a]);
                    const int na = a == 0 ? nx : ny;
                    double l = ceil((m3[a] - h - origin[a]) / size[a]);
                    double u = floor((m3[a] + h - origin[a]) / size[a]);
                    lo[a] = l < 0 ? 0 : (l > na ? na : (int)l);
                    hi[a] = u > na - 1 ? na - 1 : (u < -1 ? -1 : (int)u);
                }
            }
            for (int j = lo[1]; j <= hi[1]; j++)
                for (int i = lo[0]; i <= hi[0]; i++) {
                    const double d[3] = { origin[0] + i * size[0] - m3[0], origin[1] + j * size[1] - m3[1],
                                          z - m3[2] };
                    double md = 0.0;
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++) md += d[a] * P[g][a][b] * d[b];
                    const double f = og_kern == 1 ? rho[g] * (md < OG_KAPPA2 ? 1.0 - md / OG_KAPPA2 : 0.0)
                                                  : rho[g] * exp(-0.5 * md);
                    const int64_t x = ((int64_t)kz * ny + j) * nx + i;
                    og_accum(f, md, cut2, band, V + x, Vlo + x, Vhi + x);
                }
        }
    }
    free(Sig); free(P);
}

/* ------------------------------------------------------------------ */
/* FP32 replica of the culling predicate (bit-exact specification)     */
/* Built with -ffp-contract=off: every + - * / sqrt below is one IEEE  */
/* binary32 operation, evaluated in the written order.                 */
/* ------------------------------------------------------------------ */

/* e^x by Cody-Waite reduction x = n ln2 + r and a degree-7 Taylor
 * polynomial of e^r, |r| <= ln2/2 (truncation < 6e-9 relative) */
static float og32_exp(float x)
{
    const float LOG2E = 0x1.715476p+0f;
    const float LN2_HI = 0x1.62e4p-1f;     /* ln 2 truncated to 15 significant bits */
    const float LN2_LO = 0x1.7f7d1cp-20f;  /* ln 2 - LN2_HI */
    float n = rintf(x * LOG2E);
    float r = (x - n * LN2_HI) - n * LN2_LO;
    float p = 0x1.a01a02p-13f;             /* 1/7! */
    p = p * r + 0x1.6c16c2p-10f;           /* 1/6! */
    p = p * r + 0x1.111112p-7f;            /* 1/5! */
    p = p * r + 0x1.555556p-5f;            /* 1/4! */
    p = p * r + 0x1.555556p-3f;            /* 1/3! */
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    return ldexpf(p, (int)n);
}

static void og32_sigma(const float *ls, const float *q, float S[6])
{
    float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    float n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
    float w, x, y, z;
    if (!(n2 > 0.0f) || !(n2 < INFINITY)) { w = 1.0f; x = y = z = 0.0f; }
    else { float nr = sqrtf(n2); w = qw / nr; x = qx / nr; y = qy / nr; z = qz / nr; }
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * ((y * y) + (z * z));
    R[0][1] = 2.0f * ((x * y) - (w * z));
    R[0][2] = 2.0f * ((x * z) + (w * y));
    R[1][0] = 2.0f * ((x * y) + (w * z));
    R[1][1] = 1.0f - 2.0f * ((x * x) + (z * z));
    R[1][2] = 2.0f * ((y * z) - (w * x));
    R[2][0] = 2.0f * ((x * z) - (w * y));
    R[2][1] = 2.0f * ((y * z) + (w * x));
    R[2][2] = 1.0f - 2.0f * ((x * x) + (y * y));
    float s0 = og32_exp(2.0f * ls[0]), s1 = og32_exp(2.0f * ls[1]), s2 = og32_exp(2.0f * ls[2]);
    const int ia[6] = { 0, 0, 0, 1, 1, 2 }, ib[6] = { 0, 1, 2, 1, 2, 2 };
    for (int e = 0; e < 6; e++) {
        int a = ia[e], b = ib[e];
        S[e] = (((R[a][0] * R[b][0]) * s0) + ((R[a][1] * R[b][1]) * s1)) + ((R[a][2] * R[b][2]) * s2);
    }
}

/* e_a^T Sigma e_b with Sigma packed as (00,01,02,11,12,22) */
static float og32_form(const float S[6], const float a[3], const float b[3])
{
    float t0 = ((S[0] * b[0]) + (S[1] * b[1])) + (S[2] * b[2]);
    float t1 = ((S[1] * b[0]) + (S[3] * b[1])) + (S[4] * b[2]);
    float t2 = ((S[2] * b[0]) + (S[4] * b[1])) + (S[5] * b[2]);
    return ((a[0] * t0) + (a[1] * t1)) + (a[2] * t2);
}

static float og32_dot(const float m[3], const float e[3])
{
    return ((m[0] * e[0]) + (m[1] * e[1])) + (m[2] * e[2]);
}

static int og32_lower(const float *tab, int n, float x)
{
    int lo = 0, hi = n;
    while (lo < hi) { int mid = (lo + hi) >> 1; if (tab[mid] >= x) hi = mid; else lo = mid + 1; }
    return lo;
}
static int og32_upper(const float *tab, int n, float x)
{
    int lo = 0, hi = n;
    while (lo < hi) { int mid = (lo + hi) >> 1; if (tab[mid] > x) hi = mid; else lo = mid + 1; }
    return lo - 1;
}

/* cone: interval along one detector axis from the K-sigma tangent planes */
static int og32_cone(float K2, float dsd, float ae, float aw, float see, float sew, float sww,
                     float *lo, float *hi)
{
    float alpha = (aw * aw) - (K2 * sww);
    if (!(alpha > 0.0f)) return 0;
    float beta = dsd * ((ae * aw) - (K2 * sew));
    float disc = ((((aw * aw) * see) - (((2.0f * ae) * aw) * sew)) + ((ae * ae) * sww))
                 - (K2 * ((see * sww) - (sew * sew)));
    if (!(disc > 0.0f)) disc = 0.0f;
    float r = dsd * sqrtf(K2 * disc);
    *lo = (beta - r) / alpha;
    *hi = (beta + r) / alpha;
    return 1;
}

/* the FP32 covariance records: Sigma packed (00,01,02,11,12,22) per Gaussian */
void or_records_fp32(int64_t n, const float *ls, const float *q, float *sig6)
{
    for (int64_t k = 0; k < n; k++) og32_sigma(ls + 3 * k, q + 4 * k, sig6 + 6 * k);
}

/* the cull constant: K^2 = 9.0625 (K = 3.0104), a margin over the 3-sigma cut */
#define OG32_CULL_K2 9.0625f

/*
 * FP32 cull of views v0 .. v1-1 and every Gaussian: pixel box (i0, i1, j0, j1)
 * of the detector pixels whose centre lies inside the bounding box of the
 * projected K-sigma ellipsoid, and count = number of tiles of tile_w x tile_h
 * pixels it touches (0 and a box of -1 when empty).  Output index =
 * (view - v0) * n + gid.
 *
 * Kinds 0 and 2 (parallel rays): u and v ranges mu.e +- sqrt(K^2 e^T Sigma e).
 * Kind 1 (cone beam): the tangent planes through the source (og32_cone).
 * Kind 3 (fully 3-D PET): the u range as for kind 2; the LOR of radial
 * position s between rings r1, r2 has direction e_w + kappa e_v with
 * kappa = dz / (2 sqrt(R^2 - s^2)), dz = (r2 - r1) pitch, and along it
 * a . x = z_mid for a = e_v - kappa e_w (z_mid its mid-height), so it can
 * meet the K-sigma ellipsoid only if z_mid lies in
 * mu.a +- sqrt(K^2 a^T Sigma a).  Over the columns i0..i1 kappa runs between
 * its values at the smallest and the largest |s| of those columns, and both
 * bounds are convex / concave in kappa, so the union of the intervals is
 * spanned by those two slopes.  The rows are ring pairs: row j holds the LOR
 * of mid-height z_j + |delta| pitch / 2 (z_j the ring heights), and rows past
 * the segment's last ring pair (j > n_rows - 1 - |delta|) hold none.  When
 * the widest column reaches the ring radius (R^2 - s^2 <= 0) every row of
 * the segment is taken.
 */
void or_cull_fp32_range(const og_geom *g, int64_t n, const float *mu, const float *ls, const float *q,
                        int tile_w, int tile_h, int v0, int v1, int32_t *rect, int32_t *count)
{
    float *ut = malloc(sizeof(float) * (size_t)(g->n_cols > 0 ? g->n_cols : 1));
    float *vt = malloc(sizeof(float) * (size_t)(g->n_rows > 0 ? g->n_rows : 1));
    for (int i = 0; i < g->n_cols; i++) ut[i] = (float)og_u(g, i);
    for (int j = 0; j < g->n_rows; j++) vt[j] = (float)og_v(g, j);
    float *sig = malloc(sizeof(float) * 6 * (size_t)(n > 0 ? n : 1));
    or_records_fp32(n, ls, q, sig);
    const float K2 = OG32_CULL_K2;
    float dso = (float)g->dso, dsd = (float)g->dsd;
    float R2 = (float)(g->radius * g->radius), pitch = (float)g->pitch_v;
    for (int v = v0; v < v1; v++) {
        double eu_d[3], ev_d[3], ew_d[3];
        og_frame(g, v, eu_d, ev_d, ew_d);
        float eu[3], ev[3], ew[3];
        for (int c = 0; c < 3; c++) { eu[c] = (float)eu_d[c]; ev[c] = (float)ev_d[c]; ew[c] = (float)ew_d[c]; }
        for (int64_t k = 0; k < n; k++) {
            const float *m = mu + 3 * k, *S = sig + 6 * k;
            float mu_u = og32_dot(m, eu), mu_v = og32_dot(m, ev);
            float ulo = -INFINITY, uhi = INFINITY, vlo = -INFINITY, vhi = INFINITY;
            if (g->kind == OG_CONE) {
                float aw = og32_dot(m, ew) + dso;
                float suu = og32_form(S, eu, eu), svv = og32_form(S, ev, ev), sww = og32_form(S, ew, ew);
                float suw = og32_form(S, eu, ew), svw = og32_form(S, ev, ew);
                float lo, hi;
                if (og32_cone(K2, dsd, mu_u, aw, suu, suw, sww, &lo, &hi)) { ulo = lo; uhi = hi; }
                if (og32_cone(K2, dsd, mu_v, aw, svv, svw, sww, &lo, &hi)) { vlo = lo; vhi = hi; }
            } else {
                float hu = sqrtf(K2 * og32_form(S, eu, eu));
                float hv = sqrtf(K2 * og32_form(S, ev, ev));
                ulo = mu_u - hu; uhi = mu_u + hu; vlo = mu_v - hv; vhi = mu_v + hv;
            }
            int i0 = og32_lower(ut, g->n_cols, ulo), i1 = og32_upper(ut, g->n_cols, uhi);
            int j0, j1;
            if (g->kind == OG_PET3D) {
                j0 = 0;
                j1 = -1;
                if (i0 <= i1) {
                    int delta = og_delta(g, v), ad = abs(delta);
                    float dz = (float)delta * pitch;
                    float zoff = (0.5f * (float)ad) * pitch;
                    float ua = ut[i0], ub = ut[i1];
                    float amin = (ua <= 0.0f && ub >= 0.0f) ? 0.0f : fminf(fabsf(ua), fabsf(ub));
                    float amax = fmaxf(fabsf(ua), fabsf(ub));
                    float h2a = R2 - amin * amin, h2b = R2 - amax * amax;
                    int last = g->n_rows - 1 - ad;
                    if (!(h2b > 0.0f)) {
                        j1 = last;
                    } else {
                        float mu_w = og32_dot(m, ew);
                        float svv = og32_form(S, ev, ev), svw = og32_form(S, ev, ew), sww = og32_form(S, ew, ew);
                        float zlo = INFINITY, zhi = -INFINITY;
                        for (int e = 0; e < 2; e++) {
                            float kap = (0.5f * dz) / sqrtf(e ? h2b : h2a);
                            float zc = mu_v - kap * mu_w;
                            float t = (svv - (2.0f * kap) * svw) + (kap * kap) * sww;
                            float half = sqrtf(fmaxf(K2 * t, 0.0f));
                            zlo = fminf(zlo, zc - half);
                            zhi = fmaxf(zhi, zc + half);
                        }
                        j0 = og32_lower(vt, g->n_rows, zlo - zoff);
                        j1 = og32_upper(vt, g->n_rows, zhi - zoff);
                        if (j1 > last) j1 = last;
                    }
                }
            } else {
                j0 = og32_lower(vt, g->n_rows, vlo);
                j1 = og32_upper(vt, g->n_rows, vhi);
            }
            int64_t x = (int64_t)(v - v0) * n + k;
            if (i0 > i1 || j0 > j1) {
                count[x] = 0;
                rect[4 * x] = rect[4 * x + 1] = rect[4 * x + 2] = rect[4 * x + 3] = -1;
            } else {
                int tx0 = i0 / tile_w, tx1 = i1 / tile_w, ty0 = j0 / tile_h, ty1 = j1 / tile_h;
                rect[4 * x] = i0; rect[4 * x + 1] = i1; rect[4 * x + 2] = j0; rect[4 * x + 3] = j1;
                count[x] = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
            }
        }
    }
    free(ut); free(vt); free(sig);
}

/* every view of the geometry (3-D PET: every (ring difference, angle)) */
void or_cull_fp32(const og_geom *g, int64_t n, const float *mu, const float *ls, const float *q,
                  int tile_w, int tile_h, int32_t *rect, int32_t *count)
{
    or_cull_fp32_range(g, n, mu, ls, q, tile_w, tile_h, 0, og_nviews(g), rect, count);
}
