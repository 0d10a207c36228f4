/*
 * flood_oracle.c -- plain FP64 CPU oracle of the local-inertial shallow-water
 * time step (Pierce et al., "Accelerating Physics Simulations with TPUs: An
 * Inundation Modeling Example", Methods, "Shallow Water Equations", Eq. 3-6).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg call this file; the GPU library never links it, includes it
 * or calls it, and it shares no code with the GPU library.
 *
 * The scheme is explicit, so the oracle is the algorithm written out in the
 * paper's order: boundary faces -> face discharges (Eq. 3) -> depths (Eq. 4),
 * one loop per stage, no blocking or fusion.  Compile with -ffp-contract=off.
 *
 * Readings where the paper is silent or garbled (each is an option shared by
 * name, not by code, with the GPU library):
 *   - Eq. 3's numerator lacks the time step; the de Almeida (2012) scheme the
 *     paper follows has it: q' = (q - g dt h_f d(h+z)/dx_i) / (1 + g dt n^2 |q| h_f^(-7/3)).
 *   - The friction norm uses the face's own component |q_i| (the flux "is
 *     integrated in time, independently at each axis").
 *   - h_f = max(h_L + z_L, h_R + z_R) - max(z_L, z_R) (the text after Eq. 3).
 *   - A face is dry (q' = 0) when h_f <= h_dry.
 *   - A negative depth is set to 0 and the removed volume booked as V_clip.
 *   - The face roughness is the mean of the two cells' n.
 *   - Manning per boundary cell (Eq. 5): bc_form 0 uses the flow area
 *     dx * h (R ~ h), giving a cell discharge dx h^(5/3) sqrt(S)/n; bc_form 1
 *     uses Eq. 5 literally with A = dx^2: dx^2 h^(2/3) sqrt(S)/n.
 *   - Inflow (Eq. 6): W by bisection, then the cell discharges are rescaled
 *     so that they sum to Q_in exactly.  Q_in(t) is interpolated linearly in
 *     the hydrograph table at the step's start time and held past its ends.
 *   - Outflow uses the boundary cell's depth at the start of the step; faces
 *     on no section are closed walls (q = 0).
 *   - Time step: in epochs of E steps, dt = min(dt_cap, alpha dx / sqrt(g h_max))
 *     from the depth at the epoch's first step (h_max = 0 gives dt_cap), or a
 *     constant dt (the paper's 0.1 s runs).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Work arrays inside a step: an allocation failure ends the process with a
 * message (this is a test oracle; the entry points that allocate whole grids
 * report failure by their return value instead). */
static double *work_alloc(size_t n, int zeroed)
{
    double *p = zeroed ? (double *)calloc(n ? n : 1, sizeof(double)) : (double *)malloc(sizeof(double) * (n ? n : 1));
    if (!p) {
        fprintf(stderr, "flood oracle: out of host memory (%zu doubles)\n", n);
        abort();
    }
    return p;
}

typedef struct {
    int32_t nx, ny;
    double dx, g, h_dry, cfl_alpha, dt_cap, dt_const;
    int32_t dt_mode;      /* 0: CFL epochs, 1: constant dt */
    int32_t epoch_steps;  /* E */
    int32_t bc_form;      /* 0: dx h^(5/3) sqrt(S)/n, 1: dx^2 h^(2/3) sqrt(S)/n */
    double theta;         /* flux weighting: 1 = Eq. 3 as printed, < 1 de Almeida's theta scheme */
    int32_t friction;     /* 0: |q| of the face's own component, 1: vector norm with the orthogonal mean */
} orc_params;

typedef struct {
    int32_t side;         /* 0 xmin, 1 xmax, 2 ymin, 3 ymax */
    int32_t kind;         /* 0 inflow, 1 outflow */
    double frac_start, frac_end;
    double slope;         /* S_in or S_out */
    const double *t_s, *q_m3s;
    int32_t n_pts;
} orc_section;

typedef struct {
    double t, dt, V_in, V_out, V_clip;
    int64_t step;
} orc_ledger;

static int n_threads = 1;
void orc_set_threads(int t) { n_threads = t < 1 ? 1 : t; }
int orc_get_threads(void) { return n_threads; }

#define H(a, j, i) (a)[(size_t)(j) * nx + (i)]
#define QX(a, j, i) (a)[(size_t)(j) * (nx + 1) + (i)]
#define QY(a, j, i) (a)[(size_t)(j) * nx + (i)]

/* Cells covered by a section along its side: [floor(fs L + 1/2), floor(fe L + 1/2)). */
void orc_section_range(const orc_params *p, const orc_section *s, int32_t *i0, int32_t *i1)
{
    int32_t L = (s->side == 0 || s->side == 1) ? p->ny : p->nx;
    int32_t a = (int32_t)floor(s->frac_start * L + 0.5);
    int32_t b = (int32_t)floor(s->frac_end * L + 0.5);
    if (a < 0) a = 0;
    if (b > L) b = L;
    if (b < a) b = a;
    *i0 = a;
    *i1 = b;
}

/* Grid cell (i, j) of the k-th cell along a section's side. */
static void side_cell(const orc_params *p, int32_t side, int32_t k, int32_t *i, int32_t *j)
{
    switch (side) {
    case 0: *i = 0; *j = k; break;
    case 1: *i = p->nx - 1; *j = k; break;
    case 2: *i = k; *j = 0; break;
    default: *i = k; *j = p->ny - 1; break;
    }
}

/* Q_in(t): linear interpolation in the hydrograph table, constant past its ends. */
double orc_hydrograph(const orc_section *s, double t)
{
    if (s->n_pts <= 0) return 0.0;
    if (t <= s->t_s[0]) return s->q_m3s[0];
    for (int32_t k = 1; k < s->n_pts; k++) {
        if (t <= s->t_s[k]) {
            double w = (t - s->t_s[k - 1]) / (s->t_s[k] - s->t_s[k - 1]);
            return s->q_m3s[k - 1] + w * (s->q_m3s[k] - s->q_m3s[k - 1]);
        }
    }
    return s->q_m3s[s->n_pts - 1];
}

/* Discharge (m^3/s) through one boundary cell of depth hh by Eq. 5. */
static double manning_cell(const orc_params *p, double hh, double slope, double n)
{
    if (p->bc_form == 0)
        return p->dx * pow(hh, 5.0 / 3.0) * sqrt(slope) / n;
    return p->dx * p->dx * pow(hh, 2.0 / 3.0) * sqrt(slope) / n;
}

/* Sum over the inflow section of the Eq. 5 discharges at water level W (Eq. 6). */
static double inflow_total(const orc_params *p, const orc_section *s, const double *z,
                           const double *n, int32_t i0, int32_t i1, double W)
{
    int32_t nx = p->nx;
    double total = 0.0;
    for (int32_t k = i0; k < i1; k++) {
        int32_t i, j;
        side_cell(p, s->side, k, &i, &j);
        double hh = W - H(z, j, i);
        if (hh > 0.0) total += manning_cell(p, hh, s->slope, H(n, j, i));
    }
    return total;
}

/*
 * Inverse Manning (Eq. 6): find the water level W at which the section's cell
 * discharges sum to Q, by bisection on [min z, min z + H] with H doubled from
 * 1 m until the sum reaches Q; stop after 200 halvings or a bracket below
 * 1e-12 m; W is the upper end of the bracket.  Each cell's discharge is then
 * scaled by Q / sum.  Writes the unit-width flux (m^2/s) of each section cell,
 * positive into the domain, to q_out[k - i0]; returns W.
 */
double orc_inflow_faces(const orc_params *p, const orc_section *s, const double *z,
                        const double *n, double Q, double *q_out)
{
    int32_t nx = p->nx, i0, i1;
    orc_section_range(p, s, &i0, &i1);
    double zmin = INFINITY;
    for (int32_t k = i0; k < i1; k++) {
        int32_t i, j;
        side_cell(p, s->side, k, &i, &j);
        if (H(z, j, i) < zmin) zmin = H(z, j, i);
    }
    if (!(Q > 0.0) || i1 <= i0) {
        for (int32_t k = i0; k < i1; k++) q_out[k - i0] = 0.0;
        return zmin;
    }
    double Hb = 1.0;
    while (inflow_total(p, s, z, n, i0, i1, zmin + Hb) < Q && Hb < 1e12) Hb *= 2.0;
    double lo = zmin, hi = zmin + Hb;
    for (int it = 0; it < 200 && hi - lo >= 1e-12; it++) {
        double mid = 0.5 * (lo + hi);
        if (inflow_total(p, s, z, n, i0, i1, mid) < Q) lo = mid;
        else hi = mid;
    }
    double W = hi;
    double total = inflow_total(p, s, z, n, i0, i1, W);
    for (int32_t k = i0; k < i1; k++) {
        int32_t i, j;
        side_cell(p, s->side, k, &i, &j);
        double hh = W - H(z, j, i);
        double w = hh > 0.0 ? manning_cell(p, hh, s->slope, H(n, j, i)) : 0.0;
        q_out[k - i0] = (w * (Q / total)) / p->dx;
    }
    return W;
}

/* Outflow: unit-width flux out of the domain at a boundary cell of depth h (Eq. 5). */
static double outflow_flux(const orc_params *p, double h, double slope, double n)
{
    if (!(h > p->h_dry)) return 0.0;
    return manning_cell(p, h, slope, n) / p->dx;
}

/*
 * Eq. 3 at one interior face between cells L (lower index) and R, with the
 * time step restored in the numerator and |q| the face's own component.
 */
/* Eq. 3 at one face.  q: the face's discharge (friction); qn: the discharge in
 * the numerator, q itself, or with theta < 1 the weighted
 * theta q + (1 - theta)/2 (q_prev + q_next) of the two neighbouring faces along
 * the same axis (de Almeida et al. 2012, cited in Methods). */
static double face_update(const orc_params *p, double dt, double q, double qn, double qmag, double hL,
                          double zL, double nL, double hR, double zR, double nR)
{
    double etaL = hL + zL, etaR = hR + zR;
    double hf = fmax(etaL, etaR) - fmax(zL, zR);
    if (!(hf > p->h_dry)) return 0.0;
    double nf = 0.5 * (nL + nR);
    double slope_term = p->g * dt * hf * (etaR - etaL) / p->dx;
    double hf_m73 = 1.0 / (hf * hf * cbrt(hf));
    double friction = p->g * dt * nf * nf * qmag * hf_m73;
    return (qn - slope_term) / (1.0 + friction);
}

/* |q| in the friction term: the face's own component (reading of Methods'
 * axis-by-axis integration), or the vector norm with the orthogonal component
 * taken as the mean of the four faces of the other axis around this face
 * (a, b: the two on the lower-index side, c, d: on the other). */
static double q_mag(const orc_params *p, double q, double a, double b, double c, double d)
{
    if (p->friction == 0) return fabs(q);
    const double qo = 0.25 * ((a + b) + (c + d));
    return sqrt(q * q + qo * qo);
}

/* Numerator discharge of a face from its own and its two neighbours' along the axis. */
static double theta_q(const orc_params *p, double q, double q_prev, double q_next)
{
    if (p->theta == 1.0) return q;
    const double w = 0.5 * (1.0 - p->theta);
    return p->theta * q + w * (q_prev + q_next);
}

/* Set every boundary face from the sections (walls elsewhere); books V_in, V_out. */
static void boundary_faces(const orc_params *p, const orc_section *secs, int32_t nsec,
                           const double *z, const double *n, const double *h, double dt,
                           double t, double *qxn, double *qyn, orc_ledger *led)
{
    int32_t nx = p->nx, ny = p->ny;
    for (int32_t j = 0; j < ny; j++) { QX(qxn, j, 0) = 0.0; QX(qxn, j, nx) = 0.0; }
    for (int32_t i = 0; i < nx; i++) { QY(qyn, 0, i) = 0.0; QY(qyn, ny, i) = 0.0; }
    for (int32_t s = 0; s < nsec; s++) {
        const orc_section *sec = &secs[s];
        int32_t i0, i1;
        orc_section_range(p, sec, &i0, &i1);
        if (i1 <= i0) continue;
        double *qb = work_alloc((size_t)(i1 - i0), 0);
        /* inward sign: +1 on xmin/ymin, -1 on xmax/ymax */
        double inward = (sec->side == 0 || sec->side == 2) ? 1.0 : -1.0;
        if (sec->kind == 0) {
            double Q = orc_hydrograph(sec, t);
            orc_inflow_faces(p, sec, z, n, Q, qb);
            if (Q > 0.0) led->V_in += dt * Q;
        } else {
            double vol = 0.0;
            for (int32_t k = i0; k < i1; k++) {
                int32_t i, j;
                side_cell(p, sec->side, k, &i, &j);
                double q = outflow_flux(p, H(h, j, i), sec->slope, H(n, j, i));
                qb[k - i0] = -q;           /* outflow: against the inward direction */
                vol += q * p->dx;
            }
            led->V_out += dt * vol;
        }
        for (int32_t k = i0; k < i1; k++) {
            double v = inward * qb[k - i0];
            switch (sec->side) {
            case 0: QX(qxn, k, 0) = v; break;
            case 1: QX(qxn, k, nx) = v; break;
            case 2: QY(qyn, 0, k) = v; break;
            default: QY(qyn, ny, k) = v; break;
            }
        }
        free(qb);
    }
}

/* Work arrays of one step (new face fluxes, per-row clip volumes). */
typedef struct {
    double *qxn, *qyn, *clip_row;
} orc_scratch;

static int scratch_alloc(const orc_params *p, orc_scratch *w)
{
    w->qxn = (double *)malloc(sizeof(double) * (size_t)p->ny * (p->nx + 1));
    w->qyn = (double *)malloc(sizeof(double) * (size_t)(p->ny + 1) * p->nx);
    w->clip_row = (double *)calloc((size_t)p->ny, sizeof(double));
    return (w->qxn && w->qyn && w->clip_row) ? 0 : -1;
}

static void scratch_free(orc_scratch *w)
{
    free(w->qxn);
    free(w->qyn);
    free(w->clip_row);
}

static void step_with(const orc_params *p, const orc_section *secs, int32_t nsec,
                      const double *z, const double *n, double *h, double *qx, double *qy,
                      double dt, double t, orc_ledger *led, orc_scratch *w)
{
    int32_t nx = p->nx, ny = p->ny;
    double *qxn = w->qxn, *qyn = w->qyn, *clip_row = w->clip_row;

    boundary_faces(p, secs, nsec, z, n, h, dt, t, qxn, qyn, led);

#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (int32_t j = 0; j < ny; j++)
        for (int32_t i = 1; i < nx; i++)
            QX(qxn, j, i) = face_update(p, dt, QX(qx, j, i),
                                        theta_q(p, QX(qx, j, i), QX(qx, j, i - 1), QX(qx, j, i + 1)),
                                        q_mag(p, QX(qx, j, i), QY(qy, j, i - 1), QY(qy, j, i),
                                              QY(qy, j + 1, i - 1), QY(qy, j + 1, i)),
                                        H(h, j, i - 1), H(z, j, i - 1), H(n, j, i - 1), H(h, j, i),
                                        H(z, j, i), H(n, j, i));
#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (int32_t j = 1; j < ny; j++)
        for (int32_t i = 0; i < nx; i++)
            QY(qyn, j, i) = face_update(p, dt, QY(qy, j, i),
                                        theta_q(p, QY(qy, j, i), QY(qy, j - 1, i), QY(qy, j + 1, i)),
                                        q_mag(p, QY(qy, j, i), QX(qx, j - 1, i), QX(qx, j - 1, i + 1),
                                              QX(qx, j, i), QX(qx, j, i + 1)),
                                        H(h, j - 1, i), H(z, j - 1, i), H(n, j - 1, i), H(h, j, i),
                                        H(z, j, i), H(n, j, i));

#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (int32_t j = 0; j < ny; j++) {
        double clip = 0.0;
        for (int32_t i = 0; i < nx; i++) {
            double div = (QX(qxn, j, i) - QX(qxn, j, i + 1)) + (QY(qyn, j, i) - QY(qyn, j + 1, i));
            double hn = H(h, j, i) + dt * div / p->dx;
            if (hn < 0.0) {
                clip += -hn * p->dx * p->dx;
                hn = 0.0;
            }
            H(h, j, i) = hn;
        }
        clip_row[j] = clip;
    }
    for (int32_t j = 0; j < ny; j++) led->V_clip += clip_row[j];
    memcpy(qx, qxn, sizeof(double) * (size_t)ny * (nx + 1));
    memcpy(qy, qyn, sizeof(double) * (size_t)(ny + 1) * nx);
}

/*
 * One time step of size dt starting at time t, in place on (h, qx, qy):
 * boundary faces, then Eq. 3 on every interior face, then Eq. 4 on every cell
 * with the new face fluxes.  Adds this step's volumes to the ledger (V_in,
 * V_out, V_clip); does not advance led->t or led->step.  Returns 0, or -1 if
 * the work arrays cannot be allocated.
 */
int orc_step(const orc_params *p, const orc_section *secs, int32_t nsec, const double *z,
             const double *n, double *h, double *qx, double *qy, double dt, double t,
             orc_ledger *led)
{
    orc_scratch w;
    if (scratch_alloc(p, &w)) { scratch_free(&w); return -1; }
    step_with(p, secs, nsec, z, n, h, qx, qy, dt, t, led, &w);
    scratch_free(&w);
    return 0;
}

/* Time-step rule: constant, or CFL from the deepest cell (Bates 2010 / de Almeida 2012). */
double orc_dt(const orc_params *p, const double *h)
{
    if (p->dt_mode == 1) return p->dt_const;
    double hmax = 0.0;
    size_t N = (size_t)p->nx * p->ny;
    for (size_t c = 0; c < N; c++)
        if (h[c] > hmax) hmax = h[c];
    if (!(hmax > 0.0)) return p->dt_cap;
    return fmin(p->dt_cap, p->cfl_alpha * p->dx / sqrt(p->g * hmax));
}

/*
 * n_steps steps.  At every step whose index is a multiple of E the time step
 * is re-chosen from the current depths.  If gauge_cells is given, the depth at
 * each gauge cell (flat index j*nx+i) after step k is written to
 * gauge_out[k*n_gauges + g].  If dt_log is given, the dt of step k goes there.
 * Returns 0, or -1 if the work arrays cannot be allocated.
 */
int orc_run(const orc_params *p, const orc_section *secs, int32_t nsec, const double *z,
            const double *n, double *h, double *qx, double *qy, int64_t n_steps,
            orc_ledger *led, const int64_t *gauge_cells, int32_t n_gauges, double *gauge_out,
            double *dt_log)
{
    int32_t E = p->epoch_steps > 0 ? p->epoch_steps : 1;
    orc_scratch w;
    if (scratch_alloc(p, &w)) { scratch_free(&w); return -1; }
    for (int64_t k = 0; k < n_steps; k++) {
        if (led->step % E == 0) led->dt = orc_dt(p, h);
        step_with(p, secs, nsec, z, n, h, qx, qy, led->dt, led->t, led, &w);
        led->t += led->dt;
        led->step += 1;
        if (dt_log) dt_log[k] = led->dt;
        if (gauge_cells)
            for (int32_t g = 0; g < n_gauges; g++) gauge_out[k * n_gauges + g] = h[gauge_cells[g]];
    }
    scratch_free(&w);
    return 0;
}

/*
 * Advance to the time t_end >= led->t: steps as in orc_run, except that the
 * step that would pass t_end is shortened to end exactly at t_end (the
 * run loop's final-step truncation); the epoch keeps its time step for any
 * steps after it.  *steps_taken gets the number of steps.  Returns 0, -1 if
 * the work arrays cannot be allocated, -2 if t_end < led->t.
 */
int orc_advance(const orc_params *p, const orc_section *secs, int32_t nsec, const double *z,
                const double *n, double *h, double *qx, double *qy, double t_end, orc_ledger *led,
                int64_t *steps_taken)
{
    if (!(t_end >= led->t)) return -2;
    int32_t E = p->epoch_steps > 0 ? p->epoch_steps : 1;
    orc_scratch w;
    if (scratch_alloc(p, &w)) { scratch_free(&w); return -1; }
    int64_t k = 0;
    while (led->t < t_end) {
        if (led->step % E == 0) led->dt = orc_dt(p, h);
        const int last = led->t + led->dt > t_end;     /* this step would pass t_end */
        const double dt = last ? t_end - led->t : led->dt;
        step_with(p, secs, nsec, z, n, h, qx, qy, dt, led->t, led, &w);
        led->t = last ? t_end : led->t + led->dt;
        led->step += 1;
        k += 1;
    }
    scratch_free(&w);
    *steps_taken = k;
    return 0;
}

/* Stored volume sum(h) dx^2 with compensated (Kahan) summation. */
double orc_volume(const orc_params *p, const double *h)
{
    size_t N = (size_t)p->nx * p->ny;
    double s = 0.0, c = 0.0;
    for (size_t k = 0; k < N; k++) {
        double y = h[k] - c;
        double t = s + y;
        c = (t - s) - y;
        s = t;
    }
    return s * p->dx * p->dx;
}

/* ------------------------------------------------------------------ adjoint
 * Reverse-mode derivative of the run above with the time-step schedule held
 * fixed (dt does not depend on n).  Non-smooth points take these branches:
 * max(eta_L, eta_R) sends its derivative to L on a tie; d|q|/dq = 0 at q = 0,
 * and for the vector norm d|q|/d(q, qo) = 0 where |q| = 0; the dry-face test,
 * the outflow dry test and the depth clip are constant masks.  The inflow W
 * solve (Eq. 6) is differentiated exactly through the implicit function
 * theorem.  All forward states are stored (no checkpoints).
 */

/* Forward values of one face of Eq. 3 in the general form
 * F = (qn - a hf (eta_r - eta_l)) / (1 + cc qmag), cc = g dt nf^2 hf^(-7/3):
 * qn the numerator discharge (theta_q), qmag the friction magnitude (q_mag),
 * qo the mean orthogonal discharge of the vector norm (0 otherwise). */
typedef struct {
    double q, qmag, qo, eta_l, eta_r, hf, nf, den, F, cc;
    int wet;
} face_fwd;

static face_fwd face_forward(const orc_params *p, double dt, double q, double qn, double qmag, double qo,
                             double hL, double zL, double nL, double hR, double zR, double nR)
{
    face_fwd f;
    f.q = q;
    f.qmag = qmag;
    f.qo = qo;
    f.eta_l = hL + zL;
    f.eta_r = hR + zR;
    f.hf = fmax(f.eta_l, f.eta_r) - fmax(zL, zR);
    f.wet = f.hf > p->h_dry;
    f.nf = 0.5 * (nL + nR);
    if (!f.wet) { f.F = 0.0; f.den = 1.0; f.cc = 0.0; return f; }
    double slope_term = p->g * dt * f.hf * (f.eta_r - f.eta_l) / p->dx;
    double hf_m73 = 1.0 / (f.hf * f.hf * cbrt(f.hf));
    f.cc = p->g * dt * f.nf * f.nf * hf_m73;
    f.den = 1.0 + f.cc * qmag;
    f.F = (qn - slope_term) / f.den;
    return f;
}

/* Pull mu (adjoint of the new face flux) back to the face's own old discharge
 * (lq), its two neighbours along the axis (lqp, lqn; theta weighting), each of
 * the four orthogonal faces of the vector norm (lo), h_L, h_R, n_L, n_R. */
static void face_reverse(const orc_params *p, double dt, const face_fwd *f, double mu, double *lq,
                         double *lqp, double *lqn, double *lo, double *lhL, double *lhR, double *lnL,
                         double *lnR)
{
    *lq = *lqp = *lqn = *lo = *lhL = *lhR = *lnL = *lnR = 0.0;
    if (!f->wet || mu == 0.0) return;
    double a = p->g * dt / p->dx;
    double th = p->theta, w = 0.5 * (1.0 - p->theta);
    /* dF/dqn = 1/den, dF/dqmag = -F cc / den */
    double dF_dqmag = -f->F * f->cc / f->den;
    double dqmag_dq, dqmag_dqo;
    if (p->friction == 0) {
        dqmag_dq = f->q > 0.0 ? 1.0 : (f->q < 0.0 ? -1.0 : 0.0);
        dqmag_dqo = 0.0;
    } else if (f->qmag > 0.0) {
        dqmag_dq = f->q / f->qmag;
        dqmag_dqo = f->qo / f->qmag;
    } else {
        dqmag_dq = dqmag_dqo = 0.0;
    }
    double fric = f->cc * f->qmag;
    double dF_dhf = (-a * (f->eta_r - f->eta_l) + f->F * (7.0 / 3.0) * fric / f->hf) / f->den;
    double dF_detal = a * f->hf / f->den;
    double dF_detar = -a * f->hf / f->den;
    double dF_dnf = -f->F * (2.0 * fric / f->nf) / f->den;
    int left_max = f->eta_l >= f->eta_r;
    *lq = mu * (th / f->den + dF_dqmag * dqmag_dq);
    if (p->theta != 1.0) *lqp = *lqn = mu * w / f->den;
    *lo = mu * dF_dqmag * dqmag_dqo * 0.25;
    *lhL = mu * (dF_detal + (left_max ? dF_dhf : 0.0));
    *lhR = mu * (dF_detar + (left_max ? 0.0 : dF_dhf));
    *lnL = mu * 0.5 * dF_dnf;
    *lnR = mu * 0.5 * dF_dnf;
}

/* The mean orthogonal discharge of the vector norm (0 for the face's own |q|). */
static double q_ortho(const orc_params *p, double a, double b, double c, double d)
{
    return p->friction == 0 ? 0.0 : 0.25 * ((a + b) + (c + d));
}

/* d(cell discharge)/d(depth) divided by the discharge: p_exp / h. */
static double manning_exponent(const orc_params *p) { return p->bc_form == 0 ? 5.0 / 3.0 : 2.0 / 3.0; }

/*
 * Reverse of one step.  In: forward state (h, qx, qy) at the step's start,
 * adjoints (lh, lqx, lqy) of the state after the step.  Out: the same arrays
 * hold the adjoints of the state at the step's start; gn accumulates dL/dn.
 */
static void orc_step_reverse(const orc_params *p, const orc_section *secs, int32_t nsec,
                             const double *z, const double *n, const double *h,
                             const double *qx, const double *qy, double dt, double t,
                             double *lh, double *lqx, double *lqy, double *gn)
{
    int32_t nx = p->nx, ny = p->ny;
    size_t NC = (size_t)nx * ny, NX = (size_t)ny * (nx + 1), NY = (size_t)(ny + 1) * nx;
    double *qxn = work_alloc(NX, 0);
    double *qyn = work_alloc(NY, 0);
    double *lhu = work_alloc(NC, 0);   /* adjoint of unclipped h' */
    double *lh_out = work_alloc(NC, 1);
    double *lqx_out = work_alloc(NX, 1);
    double *lqy_out = work_alloc(NY, 1);
    orc_ledger dummy = {0};

    /* forward recompute of the new face fluxes (as in the step) */
    boundary_faces(p, secs, nsec, z, n, h, dt, t, qxn, qyn, &dummy);
    for (int32_t j = 0; j < ny; j++)
        for (int32_t i = 1; i < nx; i++)
            QX(qxn, j, i) = face_update(p, dt, QX(qx, j, i),
                                        theta_q(p, QX(qx, j, i), QX(qx, j, i - 1), QX(qx, j, i + 1)),
                                        q_mag(p, QX(qx, j, i), QY(qy, j, i - 1), QY(qy, j, i),
                                              QY(qy, j + 1, i - 1), QY(qy, j + 1, i)),
                                        H(h, j, i - 1), H(z, j, i - 1), H(n, j, i - 1), H(h, j, i),
                                        H(z, j, i), H(n, j, i));
    for (int32_t j = 1; j < ny; j++)
        for (int32_t i = 0; i < nx; i++)
            QY(qyn, j, i) = face_update(p, dt, QY(qy, j, i),
                                        theta_q(p, QY(qy, j, i), QY(qy, j - 1, i), QY(qy, j + 1, i)),
                                        q_mag(p, QY(qy, j, i), QX(qx, j - 1, i), QX(qx, j - 1, i + 1),
                                              QX(qx, j, i), QX(qx, j, i + 1)),
                                        H(h, j - 1, i), H(z, j - 1, i), H(n, j - 1, i), H(h, j, i),
                                        H(z, j, i), H(n, j, i));

    /* Eq. 4 and the clip: h' = max(h + dt div / dx, 0) (kept when h + ... >= 0) */
    for (int32_t j = 0; j < ny; j++)
        for (int32_t i = 0; i < nx; i++) {
            double div = (QX(qxn, j, i) - QX(qxn, j, i + 1)) + (QY(qyn, j, i) - QY(qyn, j + 1, i));
            double hn = H(h, j, i) + dt * div / p->dx;
            H(lhu, j, i) = hn < 0.0 ? 0.0 : H(lh, j, i);
            H(lh_out, j, i) += H(lhu, j, i);
        }

    /* mu on every face = own adjoint + dt/dx (lambda_R - lambda_L) from Eq. 4 */
    double c = dt / p->dx;
    for (int32_t j = 0; j < ny; j++)
        for (int32_t i = 0; i <= nx; i++) {
            double mu = QX(lqx, j, i);
            if (i < nx) mu += c * H(lhu, j, i);
            if (i > 0) mu -= c * H(lhu, j, i - 1);
            QX(lqx, j, i) = mu;     /* reuse as mu */
        }
    for (int32_t j = 0; j <= ny; j++)
        for (int32_t i = 0; i < nx; i++) {
            double mu = QY(lqy, j, i);
            if (j < ny) mu += c * H(lhu, j, i);
            if (j > 0) mu -= c * H(lhu, j - 1, i);
            QY(lqy, j, i) = mu;
        }

    /* interior faces through Eq. 3 (numerator discharge and friction magnitude
       taken with the same neighbours as the forward step) */
    for (int32_t j = 0; j < ny; j++)
        for (int32_t i = 1; i < nx; i++) {
            double q = QX(qx, j, i);
            double a = QY(qy, j, i - 1), b = QY(qy, j, i), c = QY(qy, j + 1, i - 1), d = QY(qy, j + 1, i);
            face_fwd f = face_forward(p, dt, q, theta_q(p, q, QX(qx, j, i - 1), QX(qx, j, i + 1)),
                                      q_mag(p, q, a, b, c, d), q_ortho(p, a, b, c, d), H(h, j, i - 1),
                                      H(z, j, i - 1), H(n, j, i - 1), H(h, j, i), H(z, j, i), H(n, j, i));
            double lq, lqp, lqn, lo, lhL, lhR, lnL, lnR;
            face_reverse(p, dt, &f, QX(lqx, j, i), &lq, &lqp, &lqn, &lo, &lhL, &lhR, &lnL, &lnR);
            QX(lqx_out, j, i) += lq;
            QX(lqx_out, j, i - 1) += lqp;
            QX(lqx_out, j, i + 1) += lqn;
            QY(lqy_out, j, i - 1) += lo;
            QY(lqy_out, j, i) += lo;
            QY(lqy_out, j + 1, i - 1) += lo;
            QY(lqy_out, j + 1, i) += lo;
            H(lh_out, j, i - 1) += lhL;
            H(lh_out, j, i) += lhR;
            H(gn, j, i - 1) += lnL;
            H(gn, j, i) += lnR;
        }
    for (int32_t j = 1; j < ny; j++)
        for (int32_t i = 0; i < nx; i++) {
            double q = QY(qy, j, i);
            double a = QX(qx, j - 1, i), b = QX(qx, j - 1, i + 1), c = QX(qx, j, i), d = QX(qx, j, i + 1);
            face_fwd f = face_forward(p, dt, q, theta_q(p, q, QY(qy, j - 1, i), QY(qy, j + 1, i)),
                                      q_mag(p, q, a, b, c, d), q_ortho(p, a, b, c, d), H(h, j - 1, i),
                                      H(z, j - 1, i), H(n, j - 1, i), H(h, j, i), H(z, j, i), H(n, j, i));
            double lq, lqp, lqn, lo, lhL, lhR, lnL, lnR;
            face_reverse(p, dt, &f, QY(lqy, j, i), &lq, &lqp, &lqn, &lo, &lhL, &lhR, &lnL, &lnR);
            QY(lqy_out, j, i) += lq;
            QY(lqy_out, j - 1, i) += lqp;
            QY(lqy_out, j + 1, i) += lqn;
            QX(lqx_out, j - 1, i) += lo;
            QX(lqx_out, j - 1, i + 1) += lo;
            QX(lqx_out, j, i) += lo;
            QX(lqx_out, j, i + 1) += lo;
            H(lh_out, j - 1, i) += lhL;
            H(lh_out, j, i) += lhR;
            H(gn, j - 1, i) += lnL;
            H(gn, j, i) += lnR;
        }

    /* boundary faces */
    double pe = manning_exponent(p);
    for (int32_t s = 0; s < nsec; s++) {
        const orc_section *sec = &secs[s];
        int32_t i0, i1;
        orc_section_range(p, sec, &i0, &i1);
        if (i1 <= i0) continue;
        double inward = (sec->side == 0 || sec->side == 2) ? 1.0 : -1.0;
        int32_t m = i1 - i0;
        double *mu = work_alloc((size_t)m, 0);
        for (int32_t k = i0; k < i1; k++) {
            switch (sec->side) {
            case 0: mu[k - i0] = QX(lqx, k, 0); break;
            case 1: mu[k - i0] = QX(lqx, k, nx); break;
            case 2: mu[k - i0] = QY(lqy, 0, k); break;
            default: mu[k - i0] = QY(lqy, ny, k); break;
            }
        }
        if (sec->kind == 1) {
            /* face value = -inward * Phi(h_c, n_c) / dx for h_c > h_dry */
            for (int32_t k = i0; k < i1; k++) {
                int32_t i, j;
                side_cell(p, sec->side, k, &i, &j);
                double hc = H(h, j, i);
                if (!(hc > p->h_dry)) continue;
                double phi = manning_cell(p, hc, sec->slope, H(n, j, i)) / p->dx;
                double nu = -inward * mu[k - i0];
                H(lh_out, j, i) += nu * pe * phi / hc;
                H(gn, j, i) += -nu * phi / H(n, j, i);
            }
        } else {
            /* face value = inward * w_c / dx with sum_c w_c = Q (Eq. 6):
               dw_c/dn_j = -delta_cj w_c/n_c + (pe w_c / hhat_c) dW/dn_j,
               dW/dn_j = (w_j / n_j) / sum_c (pe w_c / hhat_c). */
            double Q = orc_hydrograph(sec, t);
            double *qb = work_alloc((size_t)m, 0);
            double W = orc_inflow_faces(p, sec, z, n, Q, qb);
            if (Q > 0.0) {
                double D = 0.0, Nnu = 0.0;
                for (int32_t k = i0; k < i1; k++) {
                    int32_t i, j;
                    side_cell(p, sec->side, k, &i, &j);
                    double hh = W - H(z, j, i);
                    if (!(hh > 0.0)) continue;
                    double w = qb[k - i0] * p->dx;
                    double nu = inward * mu[k - i0] / p->dx;
                    D += pe * w / hh;
                    Nnu += nu * pe * w / hh;
                }
                for (int32_t k = i0; k < i1; k++) {
                    int32_t i, j;
                    side_cell(p, sec->side, k, &i, &j);
                    double hh = W - H(z, j, i);
                    if (!(hh > 0.0)) continue;
                    double w = qb[k - i0] * p->dx;
                    double nu = inward * mu[k - i0] / p->dx;
                    H(gn, j, i) += (w / H(n, j, i)) * (Nnu / D - nu);
                }
            }
            free(qb);
        }
        free(mu);
    }

    memcpy(lh, lh_out, sizeof(double) * NC);
    memcpy(lqx, lqx_out, sizeof(double) * NX);
    memcpy(lqy, lqy_out, sizeof(double) * NY);
    free(qxn); free(qyn); free(lhu); free(lh_out); free(lqx_out); free(lqy_out);
}

/*
 * Gradient of L = sum_k sum_g dLdh[k, g] * h_g(after step k) style losses:
 * dLdh[k*n_gauges + g] is dL/d(depth at gauge g after step k).  Starts from
 * (h0, qx0, qy0) at led0 (time, step count, dt), runs n_steps forward storing
 * every state, then sweeps back.  Writes dL/dn to gn (zeroed here) and, if the
 * pointers are given, dL/d(h0, qx0, qy0).  Returns 0, or -1 on allocation
 * failure.  Covers Eq. 3 as printed and its theta-weighted and vector-norm
 * forms.
 */
int orc_adjoint(const orc_params *p, const orc_section *secs, int32_t nsec, const double *z,
                const double *n, const double *h0, const double *qx0, const double *qy0,
                const orc_ledger *led0, int64_t n_steps, const int64_t *gauge_cells,
                int32_t n_gauges, const double *dLdh, double *gn, double *lh0, double *lqx0,
                double *lqy0)
{
    int32_t nx = p->nx, ny = p->ny;
    size_t NC = (size_t)nx * ny, NX = (size_t)ny * (nx + 1), NY = (size_t)(ny + 1) * nx;
    size_t per = NC + NX + NY;
    double *store = (double *)malloc(sizeof(double) * per * (size_t)(n_steps + 1));
    double *dts = (double *)malloc(sizeof(double) * (size_t)(n_steps + 1));
    double *ts = (double *)malloc(sizeof(double) * (size_t)(n_steps + 1));
    double *lh = (double *)calloc(NC, sizeof(double));
    double *lqx = (double *)calloc(NX, sizeof(double));
    double *lqy = (double *)calloc(NY, sizeof(double));
    if (!store || !dts || !ts || !lh || !lqx || !lqy) {
        free(store); free(dts); free(ts); free(lh); free(lqx); free(lqy);
        return -1;
    }
    orc_ledger led = *led0;
    memcpy(store, h0, sizeof(double) * NC);
    memcpy(store + NC, qx0, sizeof(double) * NX);
    memcpy(store + NC + NX, qy0, sizeof(double) * NY);
    int32_t E = p->epoch_steps > 0 ? p->epoch_steps : 1;
    for (int64_t k = 0; k < n_steps; k++) {
        double *cur = store + per * (size_t)k, *nxt = store + per * (size_t)(k + 1);
        memcpy(nxt, cur, sizeof(double) * per);
        if (led.step % E == 0) led.dt = orc_dt(p, cur);
        dts[k] = led.dt;
        ts[k] = led.t;
        orc_step(p, secs, nsec, z, n, nxt, nxt + NC, nxt + NC + NX, led.dt, led.t, &led);
        led.t += led.dt;
        led.step += 1;
    }
    memset(gn, 0, sizeof(double) * NC);
    for (int64_t k = n_steps - 1; k >= 0; k--) {
        for (int32_t g = 0; g < n_gauges; g++) lh[gauge_cells[g]] += dLdh[k * n_gauges + g];
        const double *cur = store + per * (size_t)k;
        orc_step_reverse(p, secs, nsec, z, n, cur, cur + NC, cur + NC + NX, dts[k], ts[k], lh,
                         lqx, lqy, gn);
    }
    if (lh0) memcpy(lh0, lh, sizeof(double) * NC);
    if (lqx0) memcpy(lqx0, lqx, sizeof(double) * NX);
    if (lqy0) memcpy(lqy0, lqy, sizeof(double) * NY);
    free(store); free(dts); free(ts); free(lh); free(lqx); free(lqy);
    return 0;
}
