/*
 * FP64 CPU oracle for the self-consistent Yee / molecular-ensemble time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously-correct
 * restatement of the method of arXiv 2512.06173 (MaxwellLink), written from the
 * paper's equations.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA library: every quantity here is recomputed from its definition.
 *
 * Units: c = eps0 = mu0 = hbar = 1, cell edge 1 (Appendix A), dt = Courant number.
 * Staggering (Yee 1966, cited in Sec. II.A.1): E at integer steps, H at half steps;
 *   Ex(i,j,k) at (i+1/2, j, k)     Hx(i,j,k) at (i, j+1/2, k+1/2)
 *   Ey(i,j,k) at (i, j+1/2, k)     Hy(i,j,k) at (i+1/2, j, k+1/2)
 *   Ez(i,j,k) at (i, j, k+1/2)     Hz(i,j,k) at (i+1/2, j+1/2, k)
 * Arrays are (nz, ny, nx) row-major, x fastest.  Outside the grid a non-periodic
 * axis reads 0 (a PEC wall at index n); tangential E on the wall at index 0 is held
 * at 0.  Periodic axes wrap.
 *
 * One step n -> n+1 (Eq. Maxwell, Eq. E_regu, Eq. von-Neumann-tls, Eq.
 * dipole_derivative, Eq. J_mol, Eq. Polarization_mol):
 *   1. every molecule gathers Etilde_m = gamma_m * sum_cells E^n kappa_m   (Eq. E_regu_Emi)
 *   2. rho_m^n -> rho_m^{n+1} under H0 - Etilde_m . mu (held over the step), with
 *      the optional Lindblad terms                                          (Eq. von-Neumann-tls)
 *   3. mudot_m = (Tr rho^{n+1} mu - Tr rho^n mu) / dt                       (Eq. dipole_derivative)
 *   4. H^{n+1/2} = H^{n-1/2} - dt curl E^n  (CPML)                           (Eq. Maxwell b)
 *   5. J^{n+1/2} = sum_m gamma_m mudot_m kappa_m + sources; pole currents J_p^{n+1/2}
 *   6. E^{n+1} = E^n + dt/eps (curl H^{n+1/2} - J - sum_p J_p)               (Eq. Maxwell a)
 *   7. DFT accumulators (E at t=(n+1)dt, H at t=(n+1/2)dt), molecular energy.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define MAXLEV 8
#define MAXPOLE 4  /* dispersive poles per cell */

typedef struct {
    int n;
    double pos[3], sigma, gamma, decay, dephase;
    int kind, nsub;
    cplx H0[MAXLEV * MAXLEV], mu[3][MAXLEV * MAXLEV], rho[MAXLEV * MAXLEV];
    double Et[3], mudot[3], energy_sum;
} omol;

typedef struct {
    int axis, index, comp;
    double amp, omega, width, t0;
} osrc;

typedef struct {
    int axis, index, nfreq;
    double *omega;
    /* accumulators over the plane (two tangential E, two tangential H), per freq */
    cplx *E1, *E2, *H1, *H2;
} oplane;

typedef struct {
    int nx, ny, nz;
    double dt;
    int periodic[3];
    int pml[6];
    double pml_m, sigma_max, kappa_max, alpha_max;
    double *E[3], *H[3];
    double *psi[12];   /* CPML memory variables, full grid (0 outside the layers) */
    double *eps;       /* relative permittivity (eps_inf in Drude cells) */
    int npole;                 /* pole slots per cell */
    double *wp[MAXPOLE];       /* pole strength (plasma frequency) per slot and cell; 0: none */
    double *dg[MAXPOLE];       /* pole damping */
    double *w0[MAXPOLE];       /* pole resonance: 0 Drude, > 0 Lorentz */
    double *JD[MAXPOLE][3];    /* polarisation current of each pole at n-1/2 */
    double *PD[MAXPOLE][3];    /* polarisation of each pole at n */
    double *J[3];      /* scratch: molecular + source current at n+1/2 */
    /* CPML coefficients per axis: integer positions (E update) and half positions (H update) */
    double *bE[3], *cE[3], *kE[3], *bH[3], *cH[3], *kH[3];
    int nmol, capmol;
    omol *mol;
    int nsrc;
    osrc src[16];
    int nplane;
    oplane plane[16];
    long step;
    double absorbed;
    struct oadj *adj;  /* adjoint state (orc_adj_*), allocated on first use */
} osim;

static long nn(const osim *s) { return (long)s->nx * s->ny * s->nz; }
static int dimn(const osim *s, int a) { return a == 0 ? s->nx : (a == 1 ? s->ny : s->nz); }

/* flat index of a cell after applying the boundary rule; -1 if outside a wall */
static long cell(const osim *s, int i, int j, int k) {
    int c[3] = {i, j, k};
    for (int a = 0; a < 3; a++) {
        int n = dimn(s, a);
        if (c[a] < 0 || c[a] >= n) {
            if (!s->periodic[a]) return -1;
            c[a] = ((c[a] % n) + n) % n;
        }
    }
    return ((long)c[2] * s->ny + c[1]) * s->nx + c[0];
}

static double at(const osim *s, const double *f, int i, int j, int k) {
    long c = cell(s, i, j, k);
    return c < 0 ? 0.0 : f[c];
}

/* Roden-Gedney CPML profile (Taflove & Hagness, cited as the PML reference) at
 * position x along axis a.  Depth u in [0,1] grows towards the outer wall. */
static void pml_coeff(const osim *s, int a, double x, double *b, double *c, double *ik) {
    int n = dimn(s, a);
    int dl = s->pml[2 * a], dh = s->pml[2 * a + 1];
    double u = 0.0;
    if (dl > 0 && x < dl) u = (dl - x) / dl;
    else if (dh > 0 && x > n - dh) u = (x - (n - dh)) / dh;
    if (u <= 0.0) { *b = 0.0; *c = 0.0; *ik = 1.0; return; }
    double sig = s->sigma_max * pow(u, s->pml_m);
    double kap = 1.0 + (s->kappa_max - 1.0) * pow(u, s->pml_m);
    double alp = s->alpha_max * (1.0 - u);
    *b = exp(-(sig / kap + alp) * s->dt);
    *c = sig > 0.0 ? sig / (sig * kap + kap * kap * alp) * (*b - 1.0) : 0.0;
    *ik = 1.0 / kap;
}

osim *orc_create(int nx, int ny, int nz, double dt, const int *periodic, const int *pml,
                 double pml_m, double sigma_max, double kappa_max, double alpha_max,
                 const double *eps, int npole, const double *wp, const double *dg, const double *w0) {
    osim *s = (osim *)calloc(1, sizeof(osim));
    s->nx = nx; s->ny = ny; s->nz = nz; s->dt = dt;
    for (int a = 0; a < 3; a++) s->periodic[a] = periodic[a];
    for (int f = 0; f < 6; f++) s->pml[f] = pml[f];
    s->pml_m = pml_m; s->sigma_max = sigma_max; s->kappa_max = kappa_max; s->alpha_max = alpha_max;
    long N = nn(s);
    if (npole < 1 || npole > MAXPOLE) { free(s); return NULL; }
    s->npole = npole;
    for (int a = 0; a < 3; a++) {
        s->E[a] = calloc(N, sizeof(double));
        s->H[a] = calloc(N, sizeof(double));
        s->J[a] = calloc(N, sizeof(double));
    }
    for (int p = 0; p < 12; p++) s->psi[p] = calloc(N, sizeof(double));
    s->eps = malloc(N * sizeof(double));
    for (long c = 0; c < N; c++) s->eps[c] = eps ? eps[c] : 1.0;
    /* pole q of cell c at [q N + c] of wp, dg, w0 */
    for (int q = 0; q < npole; q++) {
        s->wp[q] = calloc(N, sizeof(double));
        s->dg[q] = calloc(N, sizeof(double));
        s->w0[q] = calloc(N, sizeof(double));
        for (int a = 0; a < 3; a++) {
            s->JD[q][a] = calloc(N, sizeof(double));
            s->PD[q][a] = calloc(N, sizeof(double));
        }
        for (long c = 0; c < N; c++) {
            if (wp) s->wp[q][c] = wp[q * N + c];
            if (dg) s->dg[q][c] = dg[q * N + c];
            if (w0) s->w0[q][c] = w0[q * N + c];
        }
    }
    for (int a = 0; a < 3; a++) {
        int n = dimn(s, a);
        s->bE[a] = malloc(n * sizeof(double)); s->cE[a] = malloc(n * sizeof(double));
        s->kE[a] = malloc(n * sizeof(double)); s->bH[a] = malloc(n * sizeof(double));
        s->cH[a] = malloc(n * sizeof(double)); s->kH[a] = malloc(n * sizeof(double));
        for (int i = 0; i < n; i++) {
            pml_coeff(s, a, (double)i, &s->bE[a][i], &s->cE[a][i], &s->kE[a][i]);
            pml_coeff(s, a, i + 0.5, &s->bH[a][i], &s->cH[a][i], &s->kH[a][i]);
        }
    }
    return s;
}

static void adj_free(osim *s);

void orc_destroy(osim *s) {
    if (!s) return;
    for (int a = 0; a < 3; a++) {
        free(s->E[a]); free(s->H[a]); free(s->J[a]);
        free(s->bE[a]); free(s->cE[a]); free(s->kE[a]);
        free(s->bH[a]); free(s->cH[a]); free(s->kH[a]);
    }
    for (int p = 0; p < 12; p++) free(s->psi[p]);
    for (int q = 0; q < s->npole; q++) {
        free(s->wp[q]); free(s->dg[q]); free(s->w0[q]);
        for (int a = 0; a < 3; a++) { free(s->JD[q][a]); free(s->PD[q][a]); }
    }
    free(s->eps);
    free(s->mol);
    adj_free(s);
    for (int p = 0; p < s->nplane; p++) {
        free(s->plane[p].omega); free(s->plane[p].E1); free(s->plane[p].E2);
        free(s->plane[p].H1); free(s->plane[p].H2);
    }
    free(s);
}

/* ------------------------------------------------------------------ molecules */

int orc_add_molecule(osim *s, int n, const double *pos, double sigma, double gamma,
                     double decay, double dephase, int kind, int nsub,
                     const double *H0_ri, const double *mu_ri, const double *rho_ri) {
    if (n < 2 || n > MAXLEV) return -1;
    if (s->nmol == s->capmol) {
        s->capmol = s->capmol ? 2 * s->capmol : 16;
        s->mol = realloc(s->mol, s->capmol * sizeof(omol));
    }
    omol *m = &s->mol[s->nmol];
    memset(m, 0, sizeof(*m));
    m->n = n; m->sigma = sigma; m->gamma = gamma; m->decay = decay; m->dephase = dephase;
    m->kind = kind; m->nsub = nsub < 1 ? 1 : nsub;
    for (int a = 0; a < 3; a++) m->pos[a] = pos[a];
    for (int e = 0; e < n * n; e++) {
        m->H0[e] = H0_ri[2 * e] + I * H0_ri[2 * e + 1];
        m->rho[e] = rho_ri[2 * e] + I * rho_ri[2 * e + 1];
        for (int a = 0; a < 3; a++)
            m->mu[a][e] = mu_ri[2 * (a * n * n + e)] + I * mu_ri[2 * (a * n * n + e) + 1];
    }
    return s->nmol++;
}

/* Gaussian kernel (Eq. Polarization_mol with the Gaussian choice of Sec. II.A.1):
 * along axis a the window is the 2R+2 indices starting at floor(pos)-R, R=ceil(3 sigma);
 * sample positions are i (stag=0) or i+1/2 (stag=1); the 1D weights are normalised
 * to sum 1 over the window, so the 3D sum of kappa times the cell volume is 1.  The
 * Gaussian is evaluated relative to the window's nearest sample (a common factor that
 * the normalisation removes), so a narrow kernel gives finite weights instead of 0/0. */
static int window(const omol *m, int a, int stag, int *i0, double *w) {
    int R = (int)ceil(3.0 * m->sigma);
    int W = 2 * R + 2;
    *i0 = (int)floor(m->pos[a]) - R;
    double d2[32], dmin = INFINITY;
    for (int t = 0; t < W; t++) {
        double x = (*i0 + t) + 0.5 * stag;
        double d = x - m->pos[a];
        d2[t] = d * d;
        if (d2[t] < dmin) dmin = d2[t];
    }
    double sum = 0.0;
    for (int t = 0; t < W; t++) {
        w[t] = exp(-(d2[t] - dmin) / (2.0 * m->sigma * m->sigma));
        sum += w[t];
    }
    for (int t = 0; t < W; t++) w[t] /= sum;
    return W;
}

/* Etilde_m^c = gamma_m * sum over the window of E^c(cell) kappa^c(cell)   (Eq. E_regu_Emi) */
static int gather(const osim *s, const omol *m, double *out) {
    for (int c = 0; c < 3; c++) {
        int i0[3], W[3];
        double w[3][32];
        for (int a = 0; a < 3; a++) W[a] = window(m, a, a == c ? 1 : 0, &i0[a], w[a]);
        double acc = 0.0;
        for (int tk = 0; tk < W[2]; tk++)
            for (int tj = 0; tj < W[1]; tj++)
                for (int ti = 0; ti < W[0]; ti++) {
                    long cc = cell(s, i0[0] + ti, i0[1] + tj, i0[2] + tk);
                    if (cc < 0) return -1;
                    acc += w[0][ti] * w[1][tj] * w[2][tk] * s->E[c][cc];
                }
        out[c] = m->gamma * acc;
    }
    return 0;
}

/* J^c(cell) += gamma_m * mudot_m^c * kappa^c(cell)   (Eq. J_mol with Eq. Polarization_mol) */
static int scatter(osim *s, const omol *m) {
    for (int c = 0; c < 3; c++) {
        int i0[3], W[3];
        double w[3][32];
        for (int a = 0; a < 3; a++) W[a] = window(m, a, a == c ? 1 : 0, &i0[a], w[a]);
        double amp = m->gamma * m->mudot[c];
        for (int tk = 0; tk < W[2]; tk++)
            for (int tj = 0; tj < W[1]; tj++)
                for (int ti = 0; ti < W[0]; ti++) {
                    long cc = cell(s, i0[0] + ti, i0[1] + tj, i0[2] + tk);
                    if (cc < 0) return -1;
                    s->J[c][cc] += amp * w[0][ti] * w[1][tj] * w[2][tk];
                }
    }
    return 0;
}

static void matmul(int n, const cplx *A, const cplx *B, cplx *C) {
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            cplx acc = 0;
            for (int l = 0; l < n; l++) acc += A[i * n + l] * B[l * n + j];
            C[i * n + j] = acc;
        }
}

static void dagger(int n, const cplx *A, cplx *B) {
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) B[j * n + i] = conj(A[i * n + j]);
}

/* Right-hand side of Eq. von-Neumann-tls in GKSL form:
 *   drho/dt = -i [H, rho] + sum_k ( L_k rho L_k^+ - 1/2 {L_k^+ L_k, rho} )
 * with ladder decay L_k = sqrt(decay) |k-1><k| (k = 1..n-1) and pure dephasing
 * L_k = sqrt(dephase) |k><k| (k = 0..n-1).  The operators are built as matrices and
 * multiplied out literally. */
static void lindblad_rhs(const omol *m, const cplx *H, const cplx *rho, cplx *out) {
    int n = m->n;
    cplx A[MAXLEV * MAXLEV], B[MAXLEV * MAXLEV], L[MAXLEV * MAXLEV], Ld[MAXLEV * MAXLEV];
    cplx LdL[MAXLEV * MAXLEV], T1[MAXLEV * MAXLEV], T2[MAXLEV * MAXLEV];
    matmul(n, H, rho, A);
    matmul(n, rho, H, B);
    for (int e = 0; e < n * n; e++) out[e] = -I * (A[e] - B[e]);
    for (int pass = 0; pass < 2; pass++) {
        double rate = pass == 0 ? m->decay : m->dephase;
        if (rate == 0.0) continue;
        for (int k = (pass == 0 ? 1 : 0); k < n; k++) {
            memset(L, 0, sizeof(L));
            if (pass == 0) L[(k - 1) * n + k] = sqrt(rate);
            else L[k * n + k] = sqrt(rate);
            dagger(n, L, Ld);
            matmul(n, Ld, L, LdL);
            matmul(n, L, rho, T1);
            matmul(n, T1, Ld, T2);          /* L rho L^+ */
            matmul(n, LdL, rho, A);
            matmul(n, rho, LdL, B);
            for (int e = 0; e < n * n; e++) out[e] += T2[e] - 0.5 * (A[e] + B[e]);
        }
    }
}

static void effective_h(const omol *m, const double *Et, cplx *H) {
    int n = m->n;
    for (int e = 0; e < n * n; e++)
        H[e] = m->H0[e] - (Et[0] * m->mu[0][e] + Et[1] * m->mu[1][e] + Et[2] * m->mu[2][e]);
}

/* exp(-i H dt) for a 2x2 Hermitian H:
 *   e^{-i tr dt/2} [cos(W dt) I - i sin(W dt)/W (H - tr/2 I)],  W = sqrt(((a-d)/2)^2 + |b|^2) */
static void unitary2(const cplx *H, double dt, cplx *U) {
    double a = creal(H[0]), d = creal(H[3]);
    cplx b = H[1];
    double h = 0.5 * (a + d), z = 0.5 * (a - d);
    double W = sqrt(z * z + creal(b * conj(b)));
    double cw = cos(W * dt);
    double sw = W > 0 ? sin(W * dt) / W : dt;
    cplx ph = cexp(-I * h * dt);
    U[0] = ph * (cw - I * sw * z);
    U[1] = ph * (-I * sw * b);
    U[2] = ph * (-I * sw * conj(b));
    U[3] = ph * (cw + I * sw * z);
}

static void mu_expect(const omol *m, const cplx *rho, double *out) {
    int n = m->n;
    for (int a = 0; a < 3; a++) {
        cplx acc = 0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) acc += rho[i * n + j] * m->mu[a][j * n + i];
        out[a] = creal(acc);
    }
}

/* Advance one molecule over dt under the held field Et; sets mudot (Eq. dipole_derivative). */
static void molecule_advance(omol *m, const double *Et, double dt) {
    int n = m->n;
    cplx H[MAXLEV * MAXLEV];
    double mu0[3], mu1[3];
    for (int a = 0; a < 3; a++) m->Et[a] = Et[a];
    mu_expect(m, m->rho, mu0);
    effective_h(m, Et, H);
    if (m->kind == 0) {
        cplx U[4], Ud[4], T[4];
        unitary2(H, dt, U);
        dagger(2, U, Ud);
        matmul(2, U, m->rho, T);
        matmul(2, T, Ud, m->rho);
    } else {
        double h = dt / m->nsub;
        cplx k1[MAXLEV * MAXLEV], k2[MAXLEV * MAXLEV], k3[MAXLEV * MAXLEV], k4[MAXLEV * MAXLEV];
        cplx tmp[MAXLEV * MAXLEV];
        for (int sstep = 0; sstep < m->nsub; sstep++) {
            lindblad_rhs(m, H, m->rho, k1);
            for (int e = 0; e < n * n; e++) tmp[e] = m->rho[e] + 0.5 * h * k1[e];
            lindblad_rhs(m, H, tmp, k2);
            for (int e = 0; e < n * n; e++) tmp[e] = m->rho[e] + 0.5 * h * k2[e];
            lindblad_rhs(m, H, tmp, k3);
            for (int e = 0; e < n * n; e++) tmp[e] = m->rho[e] + h * k3[e];
            lindblad_rhs(m, H, tmp, k4);
            for (int e = 0; e < n * n; e++)
                m->rho[e] += h / 6.0 * (k1[e] + 2.0 * k2[e] + 2.0 * k3[e] + k4[e]);
        }
    }
    mu_expect(m, m->rho, mu1);
    for (int a = 0; a < 3; a++) m->mudot[a] = (mu1[a] - mu0[a]) / dt;
}

/* ------------------------------------------------------------------ field step */

static double src_value(const osrc *q, double t) {
    double u = (t - q->t0) / q->width;
    return q->amp * exp(-0.5 * u * u) * cos(q->omega * (t - q->t0));
}

static int pec_forced(const osim *s, int comp, int i, int j, int k) {
    /* tangential E on the wall at index 0 of a non-periodic axis */
    int idx[3] = {i, j, k};
    for (int a = 0; a < 3; a++)
        if (a != comp && !s->periodic[a] && idx[a] == 0) return 1;
    return 0;
}

int orc_step(osim *s, long nsteps) {
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const double dt = s->dt;
    long N = nn(s);
    for (long it = 0; it < nsteps; it++) {
        /* 1-3: molecules */
        for (int q = 0; q < s->nmol; q++) {
            double Et[3];
            if (gather(s, &s->mol[q], Et)) return -1;
            molecule_advance(&s->mol[q], Et, dt);
        }
        /* 4: H^{n+1/2} with CPML */
        double **E = s->E, **H = s->H, **P = s->psi;
        #pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    long c = ((long)k * ny + j) * nx + i;
                    double ex = E[0][c], ey = E[1][c], ez = E[2][c];
                    double dEz_dy = at(s, E[2], i, j + 1, k) - ez;
                    double dEy_dz = at(s, E[1], i, j, k + 1) - ey;
                    double dEx_dz = at(s, E[0], i, j, k + 1) - ex;
                    double dEz_dx = at(s, E[2], i + 1, j, k) - ez;
                    double dEy_dx = at(s, E[1], i + 1, j, k) - ey;
                    double dEx_dy = at(s, E[0], i, j + 1, k) - ex;
                    P[0][c] = s->bH[1][j] * P[0][c] + s->cH[1][j] * dEz_dy;
                    P[1][c] = s->bH[2][k] * P[1][c] + s->cH[2][k] * dEy_dz;
                    P[2][c] = s->bH[2][k] * P[2][c] + s->cH[2][k] * dEx_dz;
                    P[3][c] = s->bH[0][i] * P[3][c] + s->cH[0][i] * dEz_dx;
                    P[4][c] = s->bH[0][i] * P[4][c] + s->cH[0][i] * dEy_dx;
                    P[5][c] = s->bH[1][j] * P[5][c] + s->cH[1][j] * dEx_dy;
                    double cx = (s->kH[1][j] * dEz_dy + P[0][c]) - (s->kH[2][k] * dEy_dz + P[1][c]);
                    double cy = (s->kH[2][k] * dEx_dz + P[2][c]) - (s->kH[0][i] * dEz_dx + P[3][c]);
                    double cz = (s->kH[0][i] * dEy_dx + P[4][c]) - (s->kH[1][j] * dEx_dy + P[5][c]);
                    H[0][c] -= dt * cx;
                    H[1][c] -= dt * cy;
                    H[2][c] -= dt * cz;
                }
        /* 5: currents at n+1/2 */
        for (int a = 0; a < 3; a++) memset(s->J[a], 0, N * sizeof(double));
        for (int q = 0; q < s->nmol; q++)
            if (scatter(s, &s->mol[q])) return -1;
        double th = (s->step + 0.5) * dt;
        for (int q = 0; q < s->nsrc; q++) {
            const osrc *src = &s->src[q];
            double v = src_value(src, th);
            for (int k = 0; k < nz; k++)
                for (int j = 0; j < ny; j++)
                    for (int i = 0; i < nx; i++) {
                        int idx[3] = {i, j, k};
                        if (idx[src->axis] != src->index) continue;
                        s->J[src->comp][((long)k * ny + j) * nx + i] += v;
                    }
        }
        /* 6: E^{n+1} (Drude current from E^n first) */
        double absorbed = 0.0;
        #pragma omp parallel for schedule(static) reduction(+:absorbed)
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    long c = ((long)k * ny + j) * nx + i;
                    double hx = H[0][c], hy = H[1][c], hz = H[2][c];
                    double dHz_dy = hz - at(s, H[2], i, j - 1, k);
                    double dHy_dz = hy - at(s, H[1], i, j, k - 1);
                    double dHx_dz = hx - at(s, H[0], i, j, k - 1);
                    double dHz_dx = hz - at(s, H[2], i - 1, j, k);
                    double dHy_dx = hy - at(s, H[1], i - 1, j, k);
                    double dHx_dy = hx - at(s, H[0], i, j - 1, k);
                    P[6][c] = s->bE[1][j] * P[6][c] + s->cE[1][j] * dHz_dy;
                    P[7][c] = s->bE[2][k] * P[7][c] + s->cE[2][k] * dHy_dz;
                    P[8][c] = s->bE[2][k] * P[8][c] + s->cE[2][k] * dHx_dz;
                    P[9][c] = s->bE[0][i] * P[9][c] + s->cE[0][i] * dHz_dx;
                    P[10][c] = s->bE[0][i] * P[10][c] + s->cE[0][i] * dHy_dx;
                    P[11][c] = s->bE[1][j] * P[11][c] + s->cE[1][j] * dHx_dy;
                    double curl[3];
                    curl[0] = (s->kE[1][j] * dHz_dy + P[6][c]) - (s->kE[2][k] * dHy_dz + P[7][c]);
                    curl[1] = (s->kE[2][k] * dHx_dz + P[8][c]) - (s->kE[0][i] * dHz_dx + P[9][c]);
                    curl[2] = (s->kE[0][i] * dHy_dx + P[10][c]) - (s->kE[1][j] * dHx_dy + P[11][c]);
                    for (int a = 0; a < 3; a++) {
                        /* each pole's ADE dJ/dt + g J + w0^2 P = wp^2 E, dP/dt = J (w0 = 0:
                           Drude), J centred at n: J^{n+1/2} from J^{n-1/2}, E^n and P^n */
                        double jp[MAXPOLE], jd = 0.0;
                        for (int q = 0; q < s->npole; q++) {
                            jp[q] = 0.0;
                            if (s->wp[q][c] == 0.0) continue;
                            double g2 = 0.5 * s->dg[q][c] * dt;
                            jp[q] = ((1.0 - g2) * s->JD[q][a][c] +
                                     dt * (s->wp[q][c] * s->wp[q][c] * E[a][c] -
                                           s->w0[q][c] * s->w0[q][c] * s->PD[q][a][c])) /
                                    (1.0 + g2);
                            jd += jp[q];
                        }
                        double e_old = E[a][c];
                        double e_new = pec_forced(s, a, i, j, k)
                                           ? 0.0
                                           : e_old + dt / s->eps[c] * (curl[a] - s->J[a][c] - jd);
                        for (int q = 0; q < s->npole; q++) {
                            if (s->wp[q][c] == 0.0) continue;
                            absorbed += jp[q] * 0.5 * (e_old + e_new) * dt;
                            s->JD[q][a][c] = jp[q];
                            if (s->w0[q][c] != 0.0) s->PD[q][a][c] += dt * jp[q];  /* P^{n+1} */
                        }
                        E[a][c] = e_new;
                    }
                }
        s->absorbed += absorbed;
        /* 7: DFT accumulators and molecular energy */
        double tE = (s->step + 1) * dt;
        for (int p = 0; p < s->nplane; p++) {
            oplane *pl = &s->plane[p];
            int a = pl->axis, b = (a + 1) % 3, c2 = (a + 2) % 3;
            int nb = dimn(s, b), nc = dimn(s, c2);
            for (int f = 0; f < pl->nfreq; f++) {
                cplx pe = cexp(I * pl->omega[f] * tE) * dt;
                cplx ph = cexp(I * pl->omega[f] * th) * dt;
                for (int v = 0; v < nc; v++)
                    for (int u = 0; u < nb; u++) {
                        int idx[3], idm[3];
                        idx[a] = pl->index; idx[b] = u; idx[c2] = v;
                        idm[a] = pl->index - 1; idm[b] = u; idm[c2] = v;
                        long o = ((long)f * nc + v) * nb + u;
                        pl->E1[o] += pe * at(s, E[b], idx[0], idx[1], idx[2]);
                        pl->E2[o] += pe * at(s, E[c2], idx[0], idx[1], idx[2]);
                        pl->H1[o] += ph * 0.5 * (at(s, H[b], idx[0], idx[1], idx[2]) +
                                                 at(s, H[b], idm[0], idm[1], idm[2]));
                        pl->H2[o] += ph * 0.5 * (at(s, H[c2], idx[0], idx[1], idx[2]) +
                                                 at(s, H[c2], idm[0], idm[1], idm[2]));
                    }
            }
        }
        for (int q = 0; q < s->nmol; q++) {
            omol *m = &s->mol[q];
            cplx acc = 0;
            for (int i = 0; i < m->n; i++)
                for (int j = 0; j < m->n; j++) acc += m->rho[i * m->n + j] * m->H0[j * m->n + i];
            m->energy_sum += creal(acc);
        }
        s->step++;
    }
    return 0;
}

/* ------------------------------------------------------------------ sources, planes */

int orc_add_source(osim *s, int axis, int index, int comp, double amp, double omega,
                   double width, double t0) {
    if (s->nsrc >= 16) return -1;
    osrc *q = &s->src[s->nsrc];
    q->axis = axis; q->index = index; q->comp = comp;
    q->amp = amp; q->omega = omega; q->width = width; q->t0 = t0;
    return s->nsrc++;
}

int orc_add_plane(osim *s, int axis, int index, int nfreq, const double *omega) {
    if (s->nplane >= 16) return -1;
    oplane *p = &s->plane[s->nplane];
    p->axis = axis; p->index = index; p->nfreq = nfreq;
    p->omega = malloc(nfreq * sizeof(double));
    memcpy(p->omega, omega, nfreq * sizeof(double));
    int b = (axis + 1) % 3, c = (axis + 2) % 3;
    long cnt = (long)nfreq * dimn(s, b) * dimn(s, c);
    p->E1 = calloc(cnt, sizeof(cplx)); p->E2 = calloc(cnt, sizeof(cplx));
    p->H1 = calloc(cnt, sizeof(cplx)); p->H2 = calloc(cnt, sizeof(cplx));
    return s->nplane++;
}

/* Net flux Re sum over the plane of (Etilde x Htilde*) . n per frequency, with
 * (a,b,c) cyclic: S_a = E_b H_c^* - E_c H_b^*; H is the mean of the two half cells
 * on either side of the plane. */
int orc_flux(const osim *s, int p, double *out) {
    if (p < 0 || p >= s->nplane) return -1;
    const oplane *pl = &s->plane[p];
    int b = (pl->axis + 1) % 3, c = (pl->axis + 2) % 3;
    long cnt = (long)dimn(s, b) * dimn(s, c);
    for (int f = 0; f < pl->nfreq; f++) {
        double acc = 0.0;
        for (long o = 0; o < cnt; o++) {
            long q = (long)f * cnt + o;
            acc += creal(pl->E1[q] * conj(pl->H2[q]) - pl->E2[q] * conj(pl->H1[q]));
        }
        out[f] = acc;
    }
    return 0;
}

/* raw plane accumulators, interleaved re/im: order E1, E2, H1, H2, each (nfreq, nc, nb) */
int orc_plane_data(const osim *s, int p, double *out) {
    if (p < 0 || p >= s->nplane) return -1;
    const oplane *pl = &s->plane[p];
    int b = (pl->axis + 1) % 3, c = (pl->axis + 2) % 3;
    long cnt = (long)pl->nfreq * dimn(s, b) * dimn(s, c);
    const cplx *arr[4] = {pl->E1, pl->E2, pl->H1, pl->H2};
    for (int q = 0; q < 4; q++)
        for (long o = 0; o < cnt; o++) {
            out[2 * (q * cnt + o)] = creal(arr[q][o]);
            out[2 * (q * cnt + o) + 1] = cimag(arr[q][o]);
        }
    return 0;
}

/* ------------------------------------------------------------------ accessors */

void orc_get_fields(const osim *s, double *out) {   /* 6 x N: Ex Ey Ez Hx Hy Hz */
    long N = nn(s);
    for (int a = 0; a < 3; a++) {
        memcpy(out + a * N, s->E[a], N * sizeof(double));
        memcpy(out + (3 + a) * N, s->H[a], N * sizeof(double));
    }
}

void orc_set_fields(osim *s, const double *in) {
    long N = nn(s);
    for (int a = 0; a < 3; a++) {
        memcpy(s->E[a], in + a * N, N * sizeof(double));
        memcpy(s->H[a], in + (3 + a) * N, N * sizeof(double));
    }
}

void orc_get_drude(const osim *s, double *out) {
    long N = nn(s);
    for (int a = 0; a < 3; a++) memcpy(out + a * N, s->JD[0][a], N * sizeof(double));
}

void orc_get_psi(const osim *s, double *out) {
    long N = nn(s);
    for (int p = 0; p < 12; p++) memcpy(out + p * N, s->psi[p], N * sizeof(double));
}

int orc_nmol(const osim *s) { return s->nmol; }

/* threads the field loops run on (OpenMP), for reporting the CPU baseline */
int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
long orc_step_count(const osim *s) { return s->step; }
double orc_absorbed(const osim *s) { return s->absorbed; }

/* per molecule: Et[3], mudot[3], energy_sum */
int orc_get_mol(const osim *s, int q, double *Et, double *mudot, double *energy_sum) {
    if (q < 0 || q >= s->nmol) return -1;
    for (int a = 0; a < 3; a++) { Et[a] = s->mol[q].Et[a]; mudot[a] = s->mol[q].mudot[a]; }
    *energy_sum = s->mol[q].energy_sum;
    return 0;
}

int orc_get_rho(const osim *s, int q, double *rho_ri) {
    if (q < 0 || q >= s->nmol) return -1;
    const omol *m = &s->mol[q];
    for (int e = 0; e < m->n * m->n; e++) {
        rho_ri[2 * e] = creal(m->rho[e]);
        rho_ri[2 * e + 1] = cimag(m->rho[e]);
    }
    return m->n;
}

int orc_set_rho(osim *s, int q, const double *rho_ri) {
    if (q < 0 || q >= s->nmol) return -1;
    omol *m = &s->mol[q];
    for (int e = 0; e < m->n * m->n; e++) m->rho[e] = rho_ri[2 * e] + I * rho_ri[2 * e + 1];
    return 0;
}

/* Field-free pieces for unit tests: gather at the current fields; advance one
 * molecule under a prescribed field (classical-path mode, Eq. E_analytical). */
int orc_gather(const osim *s, int q, double *out) {
    if (q < 0 || q >= s->nmol) return -1;
    return gather(s, &s->mol[q], out);
}

int orc_molecule_step(osim *s, int q, const double *Et, double dt, double *mudot) {
    if (q < 0 || q >= s->nmol) return -1;
    molecule_advance(&s->mol[q], Et, dt);
    for (int a = 0; a < 3; a++) mudot[a] = s->mol[q].mudot[a];
    return 0;
}

int orc_lindblad_rhs(const osim *s, int q, const double *Et, const double *rho_ri, double *out_ri) {
    if (q < 0 || q >= s->nmol) return -1;
    const omol *m = &s->mol[q];
    cplx H[MAXLEV * MAXLEV], r[MAXLEV * MAXLEV], o[MAXLEV * MAXLEV];
    for (int e = 0; e < m->n * m->n; e++) r[e] = rho_ri[2 * e] + I * rho_ri[2 * e + 1];
    effective_h(m, Et, H);
    lindblad_rhs(m, H, r, o);
    for (int e = 0; e < m->n * m->n; e++) { out_ri[2 * e] = creal(o[e]); out_ri[2 * e + 1] = cimag(o[e]); }
    return 0;
}

/* the dense molecular current of the last step (for the gather/scatter duality test) */
void orc_get_current(const osim *s, double *out) {
    long N = nn(s);
    for (int a = 0; a < 3; a++) memcpy(out + a * N, s->J[a], N * sizeof(double));
}

/* CPML coefficient tables: 6 x n (bE cE kE bH cH kH) along axis a */
void orc_pml_tables(const osim *s, int a, double *out) {
    int n = dimn(s, a);
    double *src[6] = {s->bE[a], s->cE[a], s->kE[a], s->bH[a], s->cH[a], s->kH[a]};
    for (int q = 0; q < 6; q++) memcpy(out + (long)q * n, src[q], n * sizeof(double));
}

/* ------------------------------------------------------------------ state setters */

void orc_set_psi(osim *s, const double *in) {
    long N = nn(s);
    for (int p = 0; p < 12; p++) memcpy(s->psi[p], in + p * N, N * sizeof(double));
}

void orc_set_drude(osim *s, const double *in) {
    long N = nn(s);
    for (int a = 0; a < 3; a++) memcpy(s->JD[0][a], in + a * N, N * sizeof(double));
}

/* ================================================================== adjoint
 *
 * Discrete adjoint (reverse mode) of orc_step, for gradients of a DFT-flux value
 * (the Sec. IV spectra) with respect to the permittivity of every cell and the
 * coupling gamma of every molecule.  Each forward statement
 *     y = f(x1, x2, ...)
 * is undone in reverse order by adding (df/dxi)^T ybar to xbar_i; nothing is
 * reorganised, so the code below can be read against orc_step line by line.
 * Complex matrices are real vectors under <X, Y> = Re sum conj(X_ij) Y_ij.
 * Molecules: the exact two-level propagator and the RK4 GKSL step.  Dispersive media:
 * every pole slot, Drude and Lorentz.
 */


struct oadj {
    double *Eb[3], *Hb[3], *Pb[12];  /* adjoints of E, H, psi */
    double *JDb[MAXPOLE][3], *PDb[MAXPOLE][3];  /* adjoints of each pole's current and polarisation */
    double *Jb[3];     /* adjoint of the molecular + source current of the step */
    double *Eb_in[3];  /* scratch: adjoint of E^n while a step is reversed */
    cplx *rhob;        /* nmol x MAXLEV^2: adjoint of each density matrix */
};

static void adj_free(osim *s) {
    struct oadj *A = s->adj;
    if (!A) return;
    for (int a = 0; a < 3; a++) {
        free(A->Eb[a]); free(A->Hb[a]); free(A->Jb[a]); free(A->Eb_in[a]);
        for (int q = 0; q < MAXPOLE; q++) { free(A->JDb[q][a]); free(A->PDb[q][a]); }
    }
    for (int p = 0; p < 12; p++) free(A->Pb[p]);
    free(A->rhob);
    free(A);
    s->adj = NULL;
}

/* Allocate the adjoint state, all zero. */
void orc_adj_reset(osim *s) {
    adj_free(s);
    long N = nn(s);
    struct oadj *A = calloc(1, sizeof(*A));
    for (int a = 0; a < 3; a++) {
        A->Eb[a] = calloc(N, sizeof(double)); A->Hb[a] = calloc(N, sizeof(double));
        A->Jb[a] = calloc(N, sizeof(double));
        A->Eb_in[a] = calloc(N, sizeof(double));
        for (int q = 0; q < s->npole; q++) {
            A->JDb[q][a] = calloc(N, sizeof(double));
            A->PDb[q][a] = calloc(N, sizeof(double));
        }
    }
    for (int p = 0; p < 12; p++) A->Pb[p] = calloc(N, sizeof(double));
    A->rhob = calloc((size_t)(s->nmol > 0 ? s->nmol : 1) * MAXLEV * MAXLEV, sizeof(cplx));
    s->adj = A;
}

/* adjoint field state as (18 + 6 npole) x N doubles: Eb[3], Hb[3], Pb[12], then per
 * pole slot JDb[3], PDb[3] */
void orc_adj_get(const osim *s, double *out) {
    const struct oadj *A = s->adj;
    long N = nn(s);
    for (int a = 0; a < 3; a++) {
        memcpy(out + a * N, A->Eb[a], N * sizeof(double));
        memcpy(out + (3 + a) * N, A->Hb[a], N * sizeof(double));
        for (int q = 0; q < s->npole; q++) {
            memcpy(out + (18 + 6 * q + a) * N, A->JDb[q][a], N * sizeof(double));
            memcpy(out + (21 + 6 * q + a) * N, A->PDb[q][a], N * sizeof(double));
        }
    }
    for (int p = 0; p < 12; p++) memcpy(out + (6 + p) * N, A->Pb[p], N * sizeof(double));
}

void orc_adj_set(osim *s, const double *in) {
    struct oadj *A = s->adj;
    long N = nn(s);
    for (int a = 0; a < 3; a++) {
        memcpy(A->Eb[a], in + a * N, N * sizeof(double));
        memcpy(A->Hb[a], in + (3 + a) * N, N * sizeof(double));
        for (int q = 0; q < s->npole; q++) {
            memcpy(A->JDb[q][a], in + (18 + 6 * q + a) * N, N * sizeof(double));
            memcpy(A->PDb[q][a], in + (21 + 6 * q + a) * N, N * sizeof(double));
        }
    }
    for (int p = 0; p < 12; p++) memcpy(A->Pb[p], in + (6 + p) * N, N * sizeof(double));
}

/* every pole's state as 6 npole x N doubles: per slot JD[3] (n-1/2), PD[3] (n) */
int orc_npole(const osim *s) { return s->npole; }
void orc_get_poles(const osim *s, double *out) {
    long N = nn(s);
    for (int q = 0; q < s->npole; q++)
        for (int a = 0; a < 3; a++) {
            memcpy(out + (6 * q + a) * N, s->JD[q][a], N * sizeof(double));
            memcpy(out + (6 * q + 3 + a) * N, s->PD[q][a], N * sizeof(double));
        }
}
void orc_set_poles(osim *s, const double *in) {
    long N = nn(s);
    for (int q = 0; q < s->npole; q++)
        for (int a = 0; a < 3; a++) {
            memcpy(s->JD[q][a], in + (6 * q + a) * N, N * sizeof(double));
            memcpy(s->PD[q][a], in + (6 * q + 3 + a) * N, N * sizeof(double));
        }
}

/* f(i,j,k) += v if the cell exists (the transpose of reading it through at()) */
static void adj_add(const osim *s, double *f, int i, int j, int k, double v) {
    long c = cell(s, i, j, k);
    if (c >= 0) f[c] += v;
}

/* Reverse of steps 4-6 of orc_step (CPML H update, currents, E update with the
 * dispersive poles).  On entry the state holds the adjoints of the step's outputs
 * (E^{n+1}, H^{n+1/2}, psi after the step, each pole's J^{n+1/2} and P^{n+1}); on exit
 * those of its inputs (E^n, H^{n-1/2}, psi before, J^{n-1/2}, P^n).  Jb receives the adjoint of the current J^{n+1/2}.
 * With grad_eps, adds d(objective)/d eps of every cell, which needs E^n (En) and
 * E^{n+1} (En1): dE^{n+1}/d eps = -(E^{n+1} - E^n) / eps in a cell that is not held
 * at zero. */
static void adj_field_step(osim *s, const double *En, const double *En1, double *grad_eps) {
    struct oadj *A = s->adj;
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const double dt = s->dt;
    const long N = nn(s);
    double **Eb = A->Eb, **Hb = A->Hb, **Pb = A->Pb;
    for (int a = 0; a < 3; a++) {
        memset(A->Eb_in[a], 0, N * sizeof(double));
        memset(A->Jb[a], 0, N * sizeof(double));
    }
    /* ---- step 6 reversed (E update), cell by cell */
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long c = ((long)k * ny + j) * nx + i;
                double curlb[3] = {0.0, 0.0, 0.0};
                for (int a = 0; a < 3; a++) {
                    double eb = Eb[a][c];
                    double jdb = 0.0;
                    if (!pec_forced(s, a, i, j, k)) {
                        /* e_new = e_old + dt/eps (curl - J - jd) */
                        double g = dt / s->eps[c];
                        A->Eb_in[a][c] += eb;
                        curlb[a] = g * eb;
                        A->Jb[a][c] = -g * eb;
                        jdb = -g * eb;
                        if (grad_eps) grad_eps[c] += eb * (-(En1[a * N + c] - En[a * N + c]) / s->eps[c]);
                    }
                    for (int q = 0; q < s->npole; q++) {
                        if (s->wp[q][c] == 0.0) continue;
                        /* JD_q = jp; jp = ((1 - g2) JD_old + dt (wp^2 E^n - w0^2 P^n)) / (1 + g2);
                         * P^{n+1} = P^n + dt jp (Lorentz).  Adjoint of jp: its part of the E
                         * update, the carried JD_q adjoint and, through P^{n+1}, dt Pbar */
                        double g2 = 0.5 * s->dg[q][c] * dt;
                        double tot = jdb + A->JDb[q][a][c];
                        if (s->w0[q][c] != 0.0) tot += dt * A->PDb[q][a][c];
                        A->JDb[q][a][c] = tot * (1.0 - g2) / (1.0 + g2);
                        A->Eb_in[a][c] += tot * dt * s->wp[q][c] * s->wp[q][c] / (1.0 + g2);
                        if (s->w0[q][c] != 0.0)
                            A->PDb[q][a][c] -= tot * dt * s->w0[q][c] * s->w0[q][c] / (1.0 + g2);
                    }
                }
                /* curl[0] = (kE_y dHz_dy + P6) - (kE_z dHy_dz + P7), P6 = bE_y P6 + cE_y dHz_dy, ... */
                double t6 = Pb[6][c] + curlb[0], t7 = Pb[7][c] - curlb[0];
                double t8 = Pb[8][c] + curlb[1], t9 = Pb[9][c] - curlb[1];
                double t10 = Pb[10][c] + curlb[2], t11 = Pb[11][c] - curlb[2];
                double dHz_dy = s->kE[1][j] * curlb[0] + s->cE[1][j] * t6;
                double dHy_dz = -s->kE[2][k] * curlb[0] + s->cE[2][k] * t7;
                double dHx_dz = s->kE[2][k] * curlb[1] + s->cE[2][k] * t8;
                double dHz_dx = -s->kE[0][i] * curlb[1] + s->cE[0][i] * t9;
                double dHy_dx = s->kE[0][i] * curlb[2] + s->cE[0][i] * t10;
                double dHx_dy = -s->kE[1][j] * curlb[2] + s->cE[1][j] * t11;
                Pb[6][c] = s->bE[1][j] * t6;
                Pb[7][c] = s->bE[2][k] * t7;
                Pb[8][c] = s->bE[2][k] * t8;
                Pb[9][c] = s->bE[0][i] * t9;
                Pb[10][c] = s->bE[0][i] * t10;
                Pb[11][c] = s->bE[1][j] * t11;
                /* dHz_dy = hz - H_z(i, j-1, k), ... */
                Hb[2][c] += dHz_dy; adj_add(s, Hb[2], i, j - 1, k, -dHz_dy);
                Hb[1][c] += dHy_dz; adj_add(s, Hb[1], i, j, k - 1, -dHy_dz);
                Hb[0][c] += dHx_dz; adj_add(s, Hb[0], i, j, k - 1, -dHx_dz);
                Hb[2][c] += dHz_dx; adj_add(s, Hb[2], i - 1, j, k, -dHz_dx);
                Hb[1][c] += dHy_dx; adj_add(s, Hb[1], i - 1, j, k, -dHy_dx);
                Hb[0][c] += dHx_dy; adj_add(s, Hb[0], i, j - 1, k, -dHx_dy);
            }
    /* ---- step 5: J^{n+1/2} depends on the molecules (reversed by the caller) and on
     * the sources (no parameter) */
    /* ---- step 4 reversed (H update): H_new = H_old - dt c, c from the CPML curl of E^n */
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long c = ((long)k * ny + j) * nx + i;
                double cxb = -dt * Hb[0][c], cyb = -dt * Hb[1][c], czb = -dt * Hb[2][c];
                double t0 = Pb[0][c] + cxb, t1 = Pb[1][c] - cxb;
                double t2 = Pb[2][c] + cyb, t3 = Pb[3][c] - cyb;
                double t4 = Pb[4][c] + czb, t5 = Pb[5][c] - czb;
                double dEz_dy = s->kH[1][j] * cxb + s->cH[1][j] * t0;
                double dEy_dz = -s->kH[2][k] * cxb + s->cH[2][k] * t1;
                double dEx_dz = s->kH[2][k] * cyb + s->cH[2][k] * t2;
                double dEz_dx = -s->kH[0][i] * cyb + s->cH[0][i] * t3;
                double dEy_dx = s->kH[0][i] * czb + s->cH[0][i] * t4;
                double dEx_dy = -s->kH[1][j] * czb + s->cH[1][j] * t5;
                Pb[0][c] = s->bH[1][j] * t0;
                Pb[1][c] = s->bH[2][k] * t1;
                Pb[2][c] = s->bH[2][k] * t2;
                Pb[3][c] = s->bH[0][i] * t3;
                Pb[4][c] = s->bH[0][i] * t4;
                Pb[5][c] = s->bH[1][j] * t5;
                /* dEz_dy = E_z(i, j+1, k) - ez, ... */
                adj_add(s, A->Eb_in[2], i, j + 1, k, dEz_dy); A->Eb_in[2][c] -= dEz_dy;
                adj_add(s, A->Eb_in[1], i, j, k + 1, dEy_dz); A->Eb_in[1][c] -= dEy_dz;
                adj_add(s, A->Eb_in[0], i, j, k + 1, dEx_dz); A->Eb_in[0][c] -= dEx_dz;
                adj_add(s, A->Eb_in[2], i + 1, j, k, dEz_dx); A->Eb_in[2][c] -= dEz_dx;
                adj_add(s, A->Eb_in[1], i + 1, j, k, dEy_dx); A->Eb_in[1][c] -= dEy_dx;
                adj_add(s, A->Eb_in[0], i, j + 1, k, dEx_dy); A->Eb_in[0][c] -= dEx_dy;
            }
    for (int a = 0; a < 3; a++) {
        double *t = A->Eb[a];
        A->Eb[a] = A->Eb_in[a];
        A->Eb_in[a] = t;
    }
}

/* Field part of one reversed step on the adjoint state (no molecules, no gradient). */
void orc_adj_field(osim *s) { adj_field_step(s, NULL, NULL, NULL); }

/* ---- molecules */

/* sum over the window of F^c kappa^c per component (the gather without gamma) */
static int kappa_sum(const osim *s, const omol *m, double *const F[3], double *out) {
    for (int c = 0; c < 3; c++) {
        int i0[3], W[3];
        double w[3][32];
        for (int a = 0; a < 3; a++) W[a] = window(m, a, a == c ? 1 : 0, &i0[a], w[a]);
        double acc = 0.0;
        for (int tk = 0; tk < W[2]; tk++)
            for (int tj = 0; tj < W[1]; tj++)
                for (int ti = 0; ti < W[0]; ti++) {
                    long cc = cell(s, i0[0] + ti, i0[1] + tj, i0[2] + tk);
                    if (cc < 0) return -1;
                    acc += w[0][ti] * w[1][tj] * w[2][tk] * F[c][cc];
                }
        out[c] = acc;
    }
    return 0;
}

/* F^c(cell) += amp[c] kappa^c(cell) over the window (the transpose of kappa_sum) */
static int kappa_add(const osim *s, const omol *m, double *F[3], const double *amp) {
    for (int c = 0; c < 3; c++) {
        int i0[3], W[3];
        double w[3][32];
        for (int a = 0; a < 3; a++) W[a] = window(m, a, a == c ? 1 : 0, &i0[a], w[a]);
        for (int tk = 0; tk < W[2]; tk++)
            for (int tj = 0; tj < W[1]; tj++)
                for (int ti = 0; ti < W[0]; ti++) {
                    long cc = cell(s, i0[0] + ti, i0[1] + tj, i0[2] + tk);
                    if (cc < 0) return -1;
                    F[c][cc] += amp[c] * w[0][ti] * w[1][tj] * w[2][tk];
                }
    }
    return 0;
}

/* exp(A) of a complex n x n matrix (n <= 16): scaling and squaring of the Taylor
 * series (Moler & Van Loan, "Nineteen dubious ways", method 3). */
static void expm(int n, const cplx *A, cplx *out) {
    double nrm = 0.0;
    for (int i = 0; i < n; i++) {
        double r = 0.0;
        for (int j = 0; j < n; j++) r += cabs(A[i * n + j]);
        if (r > nrm) nrm = r;
    }
    int sq = 0;
    while (nrm > 0.125) { nrm *= 0.5; sq++; }
    double sc = ldexp(1.0, -sq);
    cplx X[256], term[256], tmp[256];
    for (int e = 0; e < n * n; e++) {
        X[e] = A[e] * sc;
        out[e] = (e / n == e % n) ? 1.0 : 0.0;
        term[e] = out[e];
    }
    for (int q = 1; q <= 24; q++) {
        matmul(n, term, X, tmp);
        for (int e = 0; e < n * n; e++) {
            term[e] = tmp[e] / q;
            out[e] += term[e];
        }
    }
    for (int r = 0; r < sq; r++) {
        matmul(n, out, out, tmp);
        memcpy(out, tmp, (size_t)n * n * sizeof(cplx));
    }
}

/* Frechet derivative of exp at X in direction Ed: the upper-right block of
 * exp([[X, Ed], [0, X]]) (Van Loan 1978; Higham, Functions of Matrices, Thm 3.6). */
static void expm_frechet(int n, const cplx *X, const cplx *Ed, cplx *L) {
    int m2 = 2 * n;
    cplx B[256], EB[256];
    for (int e = 0; e < m2 * m2; e++) B[e] = 0.0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            B[i * m2 + j] = X[i * n + j];
            B[i * m2 + n + j] = Ed[i * n + j];
            B[(n + i) * m2 + n + j] = X[i * n + j];
        }
    expm(m2, B, EB);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) L[i * n + j] = EB[i * m2 + n + j];
}

static double rdot(int n, const cplx *X, const cplx *Y) {
    double acc = 0.0;
    for (int e = 0; e < n * n; e++) acc += creal(conj(X[e]) * Y[e]);
    return acc;
}

/* Adjoint of the GKSL right-hand side under the real inner product Re Tr(X^+ Y):
 * for L(rho) = -i [H, rho] + sum_k (L_k rho L_k^+ - 1/2 {L_k^+ L_k, rho}) with Hermitian H,
 *   L^+(X) = i [H, X] + sum_k (L_k^+ X L_k - 1/2 {L_k^+ L_k, X}),
 * the jump operators of lindblad_rhs, multiplied out literally. */
static void lindblad_adj(const omol *m, const cplx *H, const cplx *X, cplx *out) {
    int n = m->n;
    cplx A[MAXLEV * MAXLEV], B[MAXLEV * MAXLEV], L[MAXLEV * MAXLEV], Ld[MAXLEV * MAXLEV];
    cplx LdL[MAXLEV * MAXLEV], T1[MAXLEV * MAXLEV], T2[MAXLEV * MAXLEV];
    matmul(n, H, X, A);
    matmul(n, X, H, B);
    for (int e = 0; e < n * n; e++) out[e] = I * (A[e] - B[e]);
    for (int pass = 0; pass < 2; pass++) {
        double rate = pass == 0 ? m->decay : m->dephase;
        if (rate == 0.0) continue;
        for (int k = (pass == 0 ? 1 : 0); k < n; k++) {
            memset(L, 0, sizeof(L));
            if (pass == 0) L[(k - 1) * n + k] = sqrt(rate);
            else L[k * n + k] = sqrt(rate);
            dagger(n, L, Ld);
            matmul(n, Ld, L, LdL);
            matmul(n, Ld, X, T1);
            matmul(n, T1, L, T2);           /* L^+ X L */
            matmul(n, LdL, X, A);
            matmul(n, X, LdL, B);
            for (int e = 0; e < n * n; e++) out[e] += T2[e] - 0.5 * (A[e] + B[e]);
        }
    }
}

/* Re Tr(Y^+ dL/dEt_a (S)) for each a: H = H0 - Et . mu, so dL/dEt_a (S) = i [mu_a, S]. */
static void dl_de_dot(const omol *m, const cplx *Y, const cplx *S, double *acc) {
    int n = m->n;
    cplx A[MAXLEV * MAXLEV], B[MAXLEV * MAXLEV], D[MAXLEV * MAXLEV];
    for (int a = 0; a < 3; a++) {
        matmul(n, m->mu[a], S, A);
        matmul(n, S, m->mu[a], B);
        for (int e = 0; e < n * n; e++) D[e] = I * (A[e] - B[e]);
        acc[a] += rdot(n, Y, D);
    }
}

/* Reverse of one classic RK4 substep of length h under the held H (molecule_advance):
 * given the adjoint Y of the substep's result and its start rho, replaces Y by the
 * adjoint of rho and adds the substep's part of the adjoint of Et to Etb.  The forward
 * stages are recomputed from rho; the reverse walks them back (k4, k3, k2, k1). */
static void rk4_vjp(const omol *m, const cplx *H, const cplx *rho, double h, cplx *Y, double *Etb) {
    const int n = m->n;
    cplx k[MAXLEV * MAXLEV], S2[MAXLEV * MAXLEV], S3[MAXLEV * MAXLEV], S4[MAXLEV * MAXLEV];
    cplx kb1[MAXLEV * MAXLEV], kb2[MAXLEV * MAXLEV], kb3[MAXLEV * MAXLEV], kb4[MAXLEV * MAXLEV];
    cplx Sb[MAXLEV * MAXLEV], rb[MAXLEV * MAXLEV];
    lindblad_rhs(m, H, rho, k);
    for (int e = 0; e < n * n; e++) S2[e] = rho[e] + 0.5 * h * k[e];
    lindblad_rhs(m, H, S2, k);
    for (int e = 0; e < n * n; e++) S3[e] = rho[e] + 0.5 * h * k[e];
    lindblad_rhs(m, H, S3, k);
    for (int e = 0; e < n * n; e++) S4[e] = rho[e] + h * k[e];
    /* rho' = rho + h/6 (k1 + 2 k2 + 2 k3 + k4) */
    for (int e = 0; e < n * n; e++) {
        rb[e] = Y[e];
        kb1[e] = kb4[e] = h / 6.0 * Y[e];
        kb2[e] = kb3[e] = h / 3.0 * Y[e];
    }
    /* k4 = L(S4), S4 = rho + h k3 */
    lindblad_adj(m, H, kb4, Sb);
    dl_de_dot(m, kb4, S4, Etb);
    for (int e = 0; e < n * n; e++) { rb[e] += Sb[e]; kb3[e] += h * Sb[e]; }
    /* k3 = L(S3), S3 = rho + h/2 k2 */
    lindblad_adj(m, H, kb3, Sb);
    dl_de_dot(m, kb3, S3, Etb);
    for (int e = 0; e < n * n; e++) { rb[e] += Sb[e]; kb2[e] += 0.5 * h * Sb[e]; }
    /* k2 = L(S2), S2 = rho + h/2 k1 */
    lindblad_adj(m, H, kb2, Sb);
    dl_de_dot(m, kb2, S2, Etb);
    for (int e = 0; e < n * n; e++) { rb[e] += Sb[e]; kb1[e] += 0.5 * h * Sb[e]; }
    /* k1 = L(rho) */
    lindblad_adj(m, H, kb1, Sb);
    dl_de_dot(m, kb1, rho, Etb);
    for (int e = 0; e < n * n; e++) Y[e] = rb[e] + Sb[e];
}

/* Vector-Jacobian product of one molecule step (rho, Et) -> (rho', mudot),
 * mudot = (<mu>(rho') - <mu>(rho))/dt: given the adjoints X of rho' and mdb of mudot,
 * returns those of rho (rhob) and Et (Etb).  Exact two-level step: rho' = U rho U^+,
 * U = exp(-i dt (H0 - Et . mu)).  RK4 (kind 1): nsub classic RK4 substeps of the GKSL
 * equation, reversed substep by substep (rk4_vjp). */
static void mol_vjp_core(const omol *m, const double *Et, const cplx *rho, const cplx *X, const double *mdb,
                         double dt, cplx *rhob, double *Etb) {
    const int n = m->n;
    cplx Xt[MAXLEV * MAXLEV], H[MAXLEV * MAXLEV], A[MAXLEV * MAXLEV], U[MAXLEV * MAXLEV];
    cplx Ud[MAXLEV * MAXLEV], T1[MAXLEV * MAXLEV], T2[MAXLEV * MAXLEV];
    /* <mu_a>(r) = Re sum_ij r_ij mu_a,ji: its gradient is conj(mu_a,ji) at (i, j) */
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            cplx g = 0.0;
            for (int a = 0; a < 3; a++) g += mdb[a] / dt * conj(m->mu[a][j * n + i]);
            Xt[i * n + j] = X[i * n + j] + g;   /* total adjoint of rho' */
            rhob[i * n + j] = -g;
        }
    effective_h(m, Et, H);
    if (m->kind != 0) {
        /* forward substeps from rho (their starts kept), then the reverse */
        const int ns = m->nsub;
        const double h = dt / ns;
        cplx *st = malloc((size_t)ns * MAXLEV * MAXLEV * sizeof(cplx));
        cplx cur[MAXLEV * MAXLEV], k1[MAXLEV * MAXLEV], k2[MAXLEV * MAXLEV], k3[MAXLEV * MAXLEV];
        cplx k4[MAXLEV * MAXLEV], tmp[MAXLEV * MAXLEV];
        memcpy(cur, rho, (size_t)n * n * sizeof(cplx));
        for (int q = 0; q < ns; q++) {
            memcpy(st + (long)q * MAXLEV * MAXLEV, cur, (size_t)n * n * sizeof(cplx));
            lindblad_rhs(m, H, cur, k1);
            for (int e = 0; e < n * n; e++) tmp[e] = cur[e] + 0.5 * h * k1[e];
            lindblad_rhs(m, H, tmp, k2);
            for (int e = 0; e < n * n; e++) tmp[e] = cur[e] + 0.5 * h * k2[e];
            lindblad_rhs(m, H, tmp, k3);
            for (int e = 0; e < n * n; e++) tmp[e] = cur[e] + h * k3[e];
            lindblad_rhs(m, H, tmp, k4);
            for (int e = 0; e < n * n; e++) cur[e] += h / 6.0 * (k1[e] + 2.0 * k2[e] + 2.0 * k3[e] + k4[e]);
        }
        for (int a = 0; a < 3; a++) Etb[a] = 0.0;
        for (int q = ns - 1; q >= 0; q--) rk4_vjp(m, H, st + (long)q * MAXLEV * MAXLEV, h, Xt, Etb);
        for (int e = 0; e < n * n; e++) rhob[e] += Xt[e];
        free(st);
        return;
    }
    for (int e = 0; e < n * n; e++) A[e] = -I * dt * H[e];
    expm(n, A, U);
    dagger(n, U, Ud);
    /* rho' = U rho U^+  ->  rhob += U^+ Xt U */
    matmul(n, Ud, Xt, T1);
    matmul(n, T1, U, T2);
    for (int e = 0; e < n * n; e++) rhob[e] += T2[e];
    /* dU/dEt_a = L_exp(A, i dt mu_a) (dA/dEt_a = -i dt dH/dEt_a = i dt mu_a) */
    for (int a = 0; a < 3; a++) {
        cplx Ed[MAXLEV * MAXLEV], dU[MAXLEV * MAXLEV], dUd[MAXLEV * MAXLEV], P1[MAXLEV * MAXLEV], P2[MAXLEV * MAXLEV];
        for (int e = 0; e < n * n; e++) Ed[e] = I * dt * m->mu[a][e];
        expm_frechet(n, A, Ed, dU);
        dagger(n, dU, dUd);
        matmul(n, dU, rho, T1);
        matmul(n, T1, Ud, P1);     /* dU rho U^+ */
        matmul(n, U, rho, T1);
        matmul(n, T1, dUd, P2);    /* U rho dU^+ */
        for (int e = 0; e < n * n; e++) P1[e] += P2[e];
        Etb[a] = rdot(n, Xt, P1);
    }
}

/* The same product for molecule q at the given point (for tests): rho, X as
 * interleaved re/im n x n, mdb[3]; writes rhob (re/im) and Etb[3]. */
int orc_mol_vjp(const osim *s, int q, const double *Et, const double *rho_ri, const double *X_ri,
                const double *mdb, double *rhob_ri, double *Etb) {
    if (q < 0 || q >= s->nmol) return -1;
    const omol *m = &s->mol[q];
    int n = m->n;
    cplx rho[MAXLEV * MAXLEV], X[MAXLEV * MAXLEV], rb[MAXLEV * MAXLEV];
    for (int e = 0; e < n * n; e++) {
        rho[e] = rho_ri[2 * e] + I * rho_ri[2 * e + 1];
        X[e] = X_ri[2 * e] + I * X_ri[2 * e + 1];
    }
    mol_vjp_core(m, Et, rho, X, mdb, s->dt, rb, Etb);
    for (int e = 0; e < n * n; e++) { rhob_ri[2 * e] = creal(rb[e]); rhob_ri[2 * e + 1] = cimag(rb[e]); }
    return 0;
}

/* Reverse of steps 1-3 (and the molecular part of step 5) for molecule q at the
 * step that started from E^n (En), rho^n (rho_n), with the field Et_n and mudot md_n
 * it produced.  Uses Jb from adj_field_step and the adjoint of rho^{n+1} held in the
 * state; leaves the adjoint of rho^n there and adds gamma Etb kappa into the adjoint
 * of E^n. */
static int adj_molecule(osim *s, int q, const double *En, const cplx *rho_n, const double *Et_n,
                        const double *md_n, double *grad_gamma) {
    struct oadj *A = s->adj;
    const omol *m = &s->mol[q];
    const long N = nn(s);
    cplx *X = A->rhob + (long)q * MAXLEV * MAXLEV;
    /* step 5: J += gamma mudot kappa */
    double gJ[3], mdb[3];
    if (kappa_sum(s, m, A->Jb, gJ)) return -1;
    for (int a = 0; a < 3; a++) {
        mdb[a] = m->gamma * gJ[a];
        grad_gamma[q] += md_n[a] * gJ[a];
    }
    /* steps 2-3 */
    cplx rb[MAXLEV * MAXLEV];
    double Etb[3];
    mol_vjp_core(m, Et_n, rho_n, X, mdb, s->dt, rb, Etb);
    memcpy(X, rb, (size_t)m->n * m->n * sizeof(cplx));
    /* step 1: Et = gamma * sum E^n kappa */
    double *Fn[3] = {(double *)En, (double *)En + N, (double *)En + 2 * N};
    double G[3], amp[3];
    if (kappa_sum(s, m, Fn, G)) return -1;
    for (int a = 0; a < 3; a++) {
        grad_gamma[q] += Etb[a] * G[a];
        amp[a] = m->gamma * Etb[a];
    }
    return kappa_add(s, m, A->Eb, amp);
}

/* Objective and gradients of one run of nsteps steps from the present state.
 * Objective: the flux of plane p at frequency index f (orc_flux), counting the
 * steps of this run only (the plane's sums restart).  grad_eps (N doubles) and
 * grad_gamma (nmol doubles) receive d(objective)/d eps per cell and d/d gamma per
 * molecule.  The forward fields of every step are kept (memory 3 N (nsteps + 1)
 * doubles).  Molecules of both kinds (exact two-level, RK4 GKSL). */
int orc_adjoint_run(osim *s, long nsteps, int p, int f, double *grad_eps, double *grad_gamma, double *obj) {
    if (p < 0 || p >= s->nplane || f < 0 || f >= s->plane[p].nfreq || nsteps < 1) return -1;
    const long N = nn(s);
    const int M = s->nmol;
    const double dt = s->dt;
    oplane *pl = &s->plane[p];
    const int a = pl->axis, b = (a + 1) % 3, c2 = (a + 2) % 3;
    const int nb = dimn(s, b), nc = dimn(s, c2);
    const long cnt = (long)nb * nc;
    memset(pl->E1, 0, pl->nfreq * cnt * sizeof(cplx));
    memset(pl->E2, 0, pl->nfreq * cnt * sizeof(cplx));
    memset(pl->H1, 0, pl->nfreq * cnt * sizeof(cplx));
    memset(pl->H2, 0, pl->nfreq * cnt * sizeof(cplx));
    const long n0 = s->step;
    double *Eh = malloc((size_t)(nsteps + 1) * 3 * N * sizeof(double));
    cplx *rh = malloc((size_t)(M > 0 ? M : 1) * nsteps * MAXLEV * MAXLEV * sizeof(cplx));
    double *eth = malloc((size_t)(M > 0 ? M : 1) * nsteps * 3 * sizeof(double));
    double *mdh = malloc((size_t)(M > 0 ? M : 1) * nsteps * 3 * sizeof(double));
    if (!Eh || !rh || !eth || !mdh) { free(Eh); free(rh); free(eth); free(mdh); return -3; }
    for (int q = 0; q < 3; q++) memcpy(Eh + q * N, s->E[q], N * sizeof(double));
    int rc = 0;
    for (long n = 0; n < nsteps && rc == 0; n++) {
        for (int q = 0; q < M; q++)
            memcpy(rh + ((long)n * M + q) * MAXLEV * MAXLEV, s->mol[q].rho, MAXLEV * MAXLEV * sizeof(cplx));
        rc = orc_step(s, 1);
        for (int q = 0; q < M; q++)
            for (int c = 0; c < 3; c++) {
                eth[((long)n * M + q) * 3 + c] = s->mol[q].Et[c];
                mdh[((long)n * M + q) * 3 + c] = s->mol[q].mudot[c];
            }
        for (int q = 0; q < 3; q++) memcpy(Eh + ((n + 1) * 3 + q) * N, s->E[q], N * sizeof(double));
    }
    if (rc == 0) {
        double *fl = malloc(pl->nfreq * sizeof(double));
        orc_flux(s, p, fl);
        *obj = fl[f];
        free(fl);
        orc_adj_reset(s);
        struct oadj *A = s->adj;
        memset(grad_eps, 0, N * sizeof(double));
        if (M > 0) memset(grad_gamma, 0, M * sizeof(double));
        const double w = pl->omega[f];
        const cplx *E1 = pl->E1 + f * cnt, *E2 = pl->E2 + f * cnt, *H1 = pl->H1 + f * cnt, *H2 = pl->H2 + f * cnt;
        for (long n = nsteps - 1; n >= 0 && rc == 0; n--) {
            /* step 7 reversed: E1 += pe E_b, E2 += pe E_c at the plane, H1/H2 += ph * mean of
             * H_b/H_c over the plane and the layer below; J = Re sum (E1 H2* - E2 H1*) */
            const double S = (double)(n0 + n);
            const cplx pe = cexp(I * w * (S + 1.0) * dt) * dt;
            const cplx ph = cexp(I * w * (S + 0.5) * dt) * dt;
            for (int v = 0; v < nc; v++)
                for (int u = 0; u < nb; u++) {
                    int idx[3], idm[3];
                    idx[a] = pl->index; idx[b] = u; idx[c2] = v;
                    idm[a] = pl->index - 1; idm[b] = u; idm[c2] = v;
                    long o = (long)v * nb + u;
                    adj_add(s, A->Eb[b], idx[0], idx[1], idx[2], creal(pe * conj(H2[o])));
                    adj_add(s, A->Eb[c2], idx[0], idx[1], idx[2], -creal(pe * conj(H1[o])));
                    double hb = -0.5 * creal(E2[o] * conj(ph)), hc = 0.5 * creal(E1[o] * conj(ph));
                    adj_add(s, A->Hb[b], idx[0], idx[1], idx[2], hb);
                    adj_add(s, A->Hb[b], idm[0], idm[1], idm[2], hb);
                    adj_add(s, A->Hb[c2], idx[0], idx[1], idx[2], hc);
                    adj_add(s, A->Hb[c2], idm[0], idm[1], idm[2], hc);
                }
            adj_field_step(s, Eh + n * 3 * N, Eh + (n + 1) * 3 * N, grad_eps);
            for (int q = 0; q < M && rc == 0; q++)
                rc = adj_molecule(s, q, Eh + n * 3 * N, rh + ((long)n * M + q) * MAXLEV * MAXLEV,
                                  eth + ((long)n * M + q) * 3, mdh + ((long)n * M + q) * 3, grad_gamma);
        }
    }
    free(Eh); free(rh); free(eth); free(mdh);
    return rc;
}
