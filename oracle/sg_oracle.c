/*
 * FP64 CPU oracle for the thin-disc self-gravity field -- TEST INFRASTRUCTURE.
 *
 * This file is the plain, slow reference the CUDA path is checked against.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load it.  It shares no code with the CUDA library.
 *
 * What it computes (Rendon Restrepo et al. 2025, "Self-gravity in thin
 * protoplanetary discs 1"):
 *
 *   Sec. 2.2, Eq. "SG force kernel exact":
 *       K_ab = (1/sqrt(pi)) H_ab^-2 (d/8) e^X [K1(X) - K0(X)],  X = d^2/8,
 *       d = s / H_ab,
 *   Sec. 2.2, Eq. "mean root square height":
 *       H_ab^2 = (H_a(r')^2 + H_b(r)^2) / 2,
 *   Sec. 2.2, Eq. "volume force 2D" divided by Sigma_b (acceleration):
 *       g_b(r) = -G sum_a  integral Sigma_a(r') K_ab e_s d^2r',
 *       e_s = (r - r') / s,
 *   Sec. 5.6, Eq. "grav. potential 2D" (App. F):
 *       Phi^{ab}(r) = -G integral Sigma_a(r') e^X K0(X) / (2 sqrt(pi) H_ab) d^2r'.
 *
 * The scaled Bessel functions are evaluated from the integral representation
 * K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt (DLMF 10.32.9), so that
 *       K0e(x) = e^x K0(x)         = int_0^inf exp(-x (cosh t - 1)) dt,
 *       D(x)   = e^x (K1 - K0)(x)  = int_0^inf (cosh t - 1) exp(-x (cosh t - 1)) dt.
 * Both integrands are positive (no cancellation).  The trapezoidal rule is
 * used (exponentially convergent for these analytic, fast-decaying
 * integrands).  For x >= 1 the substitution w = 2 sqrt(x) sinh(t/2) gives
 *       K0e(x) = x^-1/2      int_0^inf exp(-w^2/2) (1 + w^2/(4x))^-1/2 dw,
 *       D(x)   = (2x^3/2)^-1 int_0^inf w^2 exp(-w^2/2) (1 + w^2/(4x))^-1/2 dw,
 * whose integrand width no longer shrinks with x.
 *
 * Discretisation (the paper is silent; reading used throughout): cell centres
 * u_i = ln r_in + (i + 1/2) du, phi_j = (j + 1/2) dphi, cell mass
 * m = Sigma r^2 du dphi (midpoint rule), self-cell excluded.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

/* w-form nodes w_n = n h_w, n = 1..NW; the Gaussian weights do not depend on x. */
#define NW 40
static const double h_w = 0.25;
static double gw[NW + 1], w2gw[NW + 1];
__attribute__((constructor)) static void init_wtab(void)
{
    for (int n = 0; n <= NW; ++n) {
        double w = n * h_w;
        gw[n] = exp(-0.5 * w * w);     /* e^-50 at n = NW: tail below 1e-22 */
        w2gw[n] = w * w * gw[n];
    }
}

static void k0e_D_one(double x, double *k0e, double *D)
{
    if (!(x > 0.0)) {            /* x = 0: both diverge; callers never pass it */
        *k0e = INFINITY;
        *D = INFINITY;
        return;
    }
    if (x >= 1.0) {
        /* w-form; the integrand's nearest singularity is at w = 2i sqrt(x), so
         * the trapezoid error is ~ exp(-4 pi sqrt(x) / h_w) <= 1e-21. */
        double s0 = 0.5, s1 = 0.0;   /* f0(0) = 1 (halved), f1(0) = 0 */
        const double q = 0.25 / x;
        for (int n = 1; n <= NW; ++n) {
            double w = n * h_w;
            double r = 1.0 / sqrt(1.0 + w * w * q);
            s0 += gw[n] * r;
            s1 += w2gw[n] * r;
        }
        *k0e = h_w * s0 / sqrt(x);
        *D = h_w * s1 / (2.0 * x * sqrt(x));
    } else {
        /* t-form; step 0.05 keeps the trapezoid error far below 1e-15. */
        const double h = 0.05;
        double s0 = 0.5, s1 = 0.0;   /* at t = 0: exp(0) = 1 (halved), (cosh-1) = 0 */
        for (int n = 1; n < 1000000; ++n) {
            double t = n * h;
            double sh = sinh(0.5 * t);
            double a = 2.0 * sh * sh;          /* cosh t - 1, cancellation free */
            double e = exp(-x * a);
            s0 += e;
            s1 += a * e;
            if (x * a > 60.0 + log1p(a)) break; /* both integrands < e^-60 */
        }
        *k0e = h * s0;
        *D = h * s1;
    }
}

/* Vectorised K0e / D for the Python driver (pins and convolution tables). */
void oracle_k0e_D(int64_t n, const double *x, double *k0e, double *D)
{
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i)
        k0e_D_one(x[i], &k0e[i], &D[i]);
}

/* Kahan-compensated accumulator. */
typedef struct { double s, c; } kahan;
static inline void kadd(kahan *k, double v)
{
    double y = v - k->c;
    double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

/*
 * Direct pair sum, one source fluid a acting on one target fluid b.
 *
 * Sources: nsrc cells at (sx, sy) with mass sm (= Sigma_a r'^2 du dphi) and
 * scale height sH (= H_a^{sg}(r')).  Targets: ntgt points (tx, ty) with
 * scale height tH (= H_b^{sg}(r)) and tskip = index of the source cell that
 * coincides with the target (the self cell, excluded), or -1.
 *
 * Adds to phi, gx, gy (Cartesian acceleration) for every target:
 *     gx,gy += -G m K e_s,    phi += -G m e^X K0(X) / (2 sqrt(pi) H_ab).
 * Pairs at zero separation are skipped as well (the kernel is singular there).
 */
void oracle_direct_pair(int64_t nsrc, const double *sx, const double *sy,
                        const double *sm, const double *sH,
                        int64_t ntgt, const double *tx, const double *ty,
                        const double *tH, const int64_t *tskip, double G,
                        double *phi, double *gx, double *gy)
{
    const double inv_sqrt_pi = 1.0 / sqrt(M_PI);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < ntgt; ++t) {
        kahan ax = {0, 0}, ay = {0, 0}, ap = {0, 0};
        const double x = tx[t], y = ty[t];
        const double Hb2 = tH[t] * tH[t];
        const int64_t skip = tskip ? tskip[t] : -1;
        for (int64_t j = 0; j < nsrc; ++j) {
            if (j == skip) continue;
            double dx = x - sx[j], dy = y - sy[j];
            double s2 = dx * dx + dy * dy;
            if (s2 == 0.0) continue;
            double s = sqrt(s2);
            double Hab2 = 0.5 * (sH[j] * sH[j] + Hb2);   /* Eq. mean root square height */
            double Hab = sqrt(Hab2);
            double d = s / Hab;
            double X = d * d / 8.0;
            double k0e, D;
            k0e_D_one(X, &k0e, &D);
            /* Eq. SG force kernel exact */
            double K = inv_sqrt_pi / Hab2 * (d / 8.0) * D;
            double f = -G * sm[j] * K / s;           /* times (r - r') gives -G m K e_s */
            kadd(&ax, f * dx);
            kadd(&ay, f * dy);
            /* Eq. grav. potential 2D */
            kadd(&ap, -G * sm[j] * k0e * 0.5 * inv_sqrt_pi / Hab);
        }
        phi[t] += ap.s;
        gx[t] += ax.s;
        gy[t] += ay.s;
    }
}
