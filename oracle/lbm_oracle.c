/*
 * Oracle (test infrastructure only): a plain, slow FP64 CPU implementation of
 * the D3Q7 lattice Boltzmann scheme for Maxwell's equations used in
 * "Radiation Forces and Torques on Janus Cylinders" (arXiv 2509.22308), Sec. III.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this file's library.  It shares no code with the CUDA path: it keeps the full
 * vector distributions (7 velocities x {e_i, h_i} x 3 components = 42 doubles per
 * site) and forms every equilibrium with generic 3-D cross products, exactly as
 * Eq. (LBGK equation) and Eq. (equilibrium distribution functions) are written.
 *
 * Readings of the paper where it is silent:
 *   - moments: D = sum_i e_i, E = D / eps_r ; B = sum_i h_i, H = B / mu_r   (Sec. III)
 *   - one step at time t: moments -> (optional Fourier accumulation of E_z, H_x,
 *     H_y with weight e^{i w t}) -> post-collision f* = 2 f^eq - f -> stream
 *     f(r + c_i, t+1) = f*_i(r, t); the +-z velocities stream onto the same
 *     (x, y) site because the fields are invariant along z.
 *   - open edges ("first-order extrapolation", Sec. III): an incoming population
 *     whose upstream site r - c_i lies outside the lattice is copied from the
 *     neighbouring interior site along its own direction, which equals the
 *     post-collision value f*_i(r, t) of the boundary site itself.
 *   - PEC cells (region III of a metallo-dielectric cylinder, Sec. II): the
 *     electric field is set to zero before both equilibria are formed.
 *   - plane-wave source at the left edge (Sec. III): the incoming +x
 *     populations at x = 0 receive the exact discrete plane wave of this lattice
 *     (dispersion relation w = (3 - z) / (z (3 z - 1)), z = e^{-i omega}); kind
 *     OPEN adds it on top of the zero-gradient copy of the scattered part, kind
 *     HARD replaces the incoming populations by the incident ones.
 *   - polarization: TM^z (E_z, H_x, H_y), the paper's case, or TE^z (H_z, E_x,
 *     E_y), which the paper leaves for future work.  The scheme is the same; only
 *     the incident wave (E_y = H_z = E0 sin(omega t - k x) instead of
 *     E_z = -H_y = E0 sin(omega t - k x)) and the reported field triple differ.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define NVEL 7               /* D3Q7: rest, +x, -x, +y, -y, +z, -z            */
#define NVEC (2 * NVEL)      /* e_0..e_6 then h_0..h_6                          */
#define SITE_DOUBLES (NVEC * 3)

static const int CV[NVEL][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

enum { SRC_OPEN = 0, SRC_HARD = 1, SRC_NONE = 2 };
enum { POL_TM = 0, POL_TE = 1 };

typedef struct {
    int nx, ny;        /* lattice size; site (x, y) is at index y * nx + x      */
    int period;        /* T: steps per period of the incident wave             */
    double E0;         /* incident amplitude                                   */
    int ramp_steps;    /* sin^2 ramp of the source over this many steps (0: none) */
    int source_kind;   /* SRC_OPEN / SRC_HARD / SRC_NONE                       */
    int nthreads;      /* OpenMP threads (<= 0: 1)                             */
    int polarization;  /* POL_TM / POL_TE                                      */
} oracle_cfg;

static void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Eq. (equilibrium distribution functions):
 *   e_i^eq = (E - c_i x H) / 6,  h_i^eq = (H + c_i x E) / 6   for i != 0
 *   e_0^eq = (eps_r - 1) E,      h_0^eq = (mu_r - 1) H                          */
void oracle_equilibria(double eps_r, double mu_r, const double E[3], const double H[3],
                       double *eeq, double *heq) {
    for (int i = 0; i < NVEL; ++i) {
        if (i == 0) {
            for (int k = 0; k < 3; ++k) {
                eeq[k] = (eps_r - 1.0) * E[k];
                heq[k] = (mu_r - 1.0) * H[k];
            }
            continue;
        }
        double c[3] = {(double)CV[i][0], (double)CV[i][1], (double)CV[i][2]};
        double cxH[3], cxE[3];
        cross3(c, H, cxH);
        cross3(c, E, cxE);
        for (int k = 0; k < 3; ++k) {
            eeq[3 * i + k] = (E[k] - cxH[k]) / 6.0;
            heq[3 * i + k] = (H[k] + cxE[k]) / 6.0;
        }
    }
}

/* Moments of one site (Sec. III, "reconstructed from the moments"). */
void oracle_site_fields(const double *site, double eps_r, int pec, double E[3], double H[3]) {
    double D[3] = {0, 0, 0}, B[3] = {0, 0, 0};
    for (int i = 0; i < NVEL; ++i)
        for (int k = 0; k < 3; ++k) {
            D[k] += site[3 * i + k];
            B[k] += site[3 * (NVEL + i) + k];
        }
    for (int k = 0; k < 3; ++k) {
        E[k] = pec ? 0.0 : D[k] / eps_r;
        H[k] = B[k] / 1.0; /* mu_r = 1 in every simulation (Sec. III) */
    }
}

/* Incident discrete plane wave: E_z(x, t) = Re[Ehat w^x z^t] with
 * Ehat = i E0, so E_z(x, t) = E0 sin(omega t - k x); the +x population of the
 * e_z component carries Re[P w^x z^t] with P = 2 Ehat / (3 (w z + 1)), the
 * y component of h_{+x} carries the negative of it.  TE: the same wave in
 * E_y = H_z, carried by the y component of e_{+x} and the z component of h_{+x}
 * (the equilibria of a wave along x only mix the populations of one transverse
 * component pair, so the one-dimensional dynamics is the same).                */
static void incident_plus_x(const oracle_cfg *cfg, long t, double *p0, double *p1) {
    const double omega = 2.0 * M_PI / (double)cfg->period;
    double complex z = cexp(-I * omega);
    double complex w = (3.0 - z) / (z * (3.0 * z - 1.0));
    double complex Ehat = I * cfg->E0;
    double complex P = 2.0 * Ehat / (3.0 * (w * z + 1.0));
    double complex zt = cexp(-I * omega * (double)(t % cfg->period));
    double ramp = 1.0;
    if (cfg->ramp_steps > 0 && t < cfg->ramp_steps) {
        double s = sin(0.5 * M_PI * (double)t / (double)cfg->ramp_steps);
        ramp = s * s;
    }
    *p0 = ramp * creal(P * zt);
    *p1 = ramp * creal(P * w * zt);
}

/* The three field components a polarization has: TM (E_z, H_x, H_y), TE (H_z, E_x, E_y). */
static void field_triple(int polarization, const double E[3], const double H[3], double out[3]) {
    if (polarization == POL_TE) {
        out[0] = H[2];
        out[1] = E[0];
        out[2] = E[1];
    } else {
        out[0] = E[2];
        out[1] = H[0];
        out[2] = H[1];
    }
}

/* The field triple of every site at the current time (TM: E_z, H_x, H_y;
 * TE: H_z, E_x, E_y). */
void oracle_fields(const oracle_cfg *cfg, const double *eps, const unsigned char *pec,
                   const double *f, double *ez, double *hx, double *hy) {
    const size_t n = (size_t)cfg->nx * (size_t)cfg->ny;
    for (size_t s = 0; s < n; ++s) {
        double E[3], H[3], v[3];
        oracle_site_fields(f + s * SITE_DOUBLES, eps[s], pec ? pec[s] : 0, E, H);
        field_triple(cfg->polarization, E, H, v);
        if (ez) ez[s] = v[0];
        if (hx) hx[s] = v[1];
        if (hy) hy[s] = v[2];
    }
}

/*
 * Advance the state f (pre-collision populations at time t0, nx*ny*42 doubles)
 * by nsteps steps.  fpost is caller scratch of the same size.  If acc is not
 * NULL, every step adds the field triple (TM: E_z, H_x, H_y; TE: H_z, E_x, E_y)
 * times (cos w t, sin w t) of every site into acc[site*6 + {0..5}].
 * Returns 0, or -1 on invalid arguments.
 */
int oracle_advance(const oracle_cfg *cfg, const double *eps, const unsigned char *pec,
                   double *f, double *fpost, long t0, long nsteps, double *acc) {
    if (!cfg || !eps || !f || !fpost || cfg->nx < 2 || cfg->ny < 2 || cfg->period < 1)
        return -1;
    const int nx = cfg->nx, ny = cfg->ny;
    const int nth = cfg->nthreads > 0 ? cfg->nthreads : 1;
    const double omega = 2.0 * M_PI / (double)cfg->period;
    const int te = cfg->polarization == POL_TE;
    (void)nth;

    for (long step = 0; step < nsteps; ++step) {
        const long t = t0 + step;
        const double cw = cos(omega * (double)(t % cfg->period));
        const double sw = sin(omega * (double)(t % cfg->period));

        /* collision: f* = 2 f^eq - f (Eq. LBGK equation) */
#pragma omp parallel for num_threads(nth) schedule(static)
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                const size_t s = (size_t)y * nx + x;
                const double *site = f + s * SITE_DOUBLES;
                double *post = fpost + s * SITE_DOUBLES;
                const int is_pec = pec ? pec[s] : 0;
                double E[3], H[3], eeq[NVEL * 3], heq[NVEL * 3];
                oracle_site_fields(site, eps[s], is_pec, E, H);
                if (acc) {
                    double *a = acc + s * 6, v[3];
                    field_triple(cfg->polarization, E, H, v);
                    a[0] += v[0] * cw; a[1] += v[0] * sw;
                    a[2] += v[1] * cw; a[3] += v[1] * sw;
                    a[4] += v[2] * cw; a[5] += v[2] * sw;
                }
                oracle_equilibria(eps[s], 1.0, E, H, eeq, heq);
                for (int j = 0; j < NVEL * 3; ++j) {
                    post[j] = 2.0 * eeq[j] - site[j];
                    post[NVEL * 3 + j] = 2.0 * heq[j] - site[NVEL * 3 + j];
                }
            }
        }

        double p0 = 0.0, p1 = 0.0;
        if (cfg->source_kind != SRC_NONE) incident_plus_x(cfg, t + 1, &p0, &p1);

        /* streaming f_i(r, t+1) = f*_i(r - c_i, t), then the edges */
#pragma omp parallel for num_threads(nth) schedule(static)
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                const size_t s = (size_t)y * nx + x;
                double *dst = f + s * SITE_DOUBLES;
                for (int i = 0; i < NVEL; ++i) {
                    const int sx = x - CV[i][0], sy = y - CV[i][1];
                    const int inside = sx >= 0 && sx < nx && sy >= 0 && sy < ny;
                    /* open edge: copy along the direction = own post-collision */
                    const size_t src = inside ? (size_t)sy * nx + sx : s;
                    for (int k = 0; k < 3; ++k) {
                        dst[3 * i + k] = fpost[src * SITE_DOUBLES + 3 * i + k];
                        dst[3 * (NVEL + i) + k] =
                            fpost[src * SITE_DOUBLES + 3 * (NVEL + i) + k];
                    }
                    /* incident +x pair: TM e_+x,z = P, h_+x,y = -P; TE e_+x,y = P, h_+x,z = P */
                    const int ek = te ? 1 : 2, hk = te ? 2 : 1;
                    const double hs = te ? 1.0 : -1.0;
                    if (x == 0 && i == 1 && cfg->source_kind == SRC_OPEN) {
                        /* scattered part extrapolated, incident part exact */
                        dst[3 * 1 + ek] += p0 - p1;
                        dst[3 * (NVEL + 1) + hk] += hs * (p0 - p1);
                    } else if (x == 0 && i == 1 && cfg->source_kind == SRC_HARD) {
                        for (int k = 0; k < 3; ++k) {
                            dst[3 * 1 + k] = 0.0;
                            dst[3 * (NVEL + 1) + k] = 0.0;
                        }
                        dst[3 * 1 + ek] = p0;
                        dst[3 * (NVEL + 1) + hk] = hs * p0;
                    }
                }
            }
        }
    }
    return 0;
}

int oracle_site_doubles(void) { return SITE_DOUBLES; }
