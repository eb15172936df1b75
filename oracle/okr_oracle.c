/*
 * okr_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU oracle for the exhaustive Kron-based reduction of an
 * unbalanced three-phase radial feeder (arXiv 2510.19608, "Optimal Kron-based
 * reduction of three-phase distribution feeders").  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header or table with the CUDA library.
 *
 * Conventions
 *   bus 0 is the substation (slack); parent[i] < i; phases are bit masks
 *   (a=1, b=2, c=4) with phases[i] a subset of phases[parent[i]].
 *   Per-bus three-phase vectors are stored padded: x[bus][3] (absent phases 0).
 *   Complex numbers are C99 `double complex` (layout = two doubles).
 *
 * Contents
 *   orc_ybus          dense compact admittance Y (Sec. II-A, eq. KCL-3phase)
 *   orc_injection     I = Y V, bus by bus (Sec. II-A)
 *   orc_pf            backward/forward-sweep AC load flow, constant-power loads
 *                     (the operating points of Sec. III; the paper does not
 *                     name its load-flow method)
 *   orc_tree_*        Gaussian elimination of the non-slack rows of Y in
 *                     leaf-first order, and the solve Y_LL V_L = I_L - Y_L0 V_0
 *   orc_zbus          Z = Y_LL^{-1}, one solve per unit injection
 *   orc_kron          Y_Kron by eliminating every reduced bus (all its phases at
 *                     once), Sec. II-B eqs. (Y-partitioned), (Y_kron)
 *   orc_reduce        Algorithm 1 (Sec. IV) in literal mode (one full solve per
 *                     candidate) or delta mode (V^c = V + (Z_s - Z_r) I_r,
 *                     the same solve by linearity)
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *   slack: bus 0 keeps V_slack, only the non-slack rows are solved, bus 0 is
 *   never reduced (it may absorb a neighbour); clusters of a candidate are the
 *   post-merge clusters (all of r's cluster moves to s and takes V^c_s); the
 *   error is per phase, e = | |Vhat| - |V^c| |; SMICE is summed over scenarios
 *   and clusters; ties: every feasible candidate with score <= min + tau is
 *   tied and the smallest (r, s) bus pair wins.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;


static double mag(cplx v) {
    double re = creal(v), im = cimag(v);
    return sqrt(re * re + im * im);
}

/* z[bus][3][3][2] -> complex */
static cplx zat(const double *z, int bus, int p, int q) {
    const double *e = z + (((size_t)bus * 3 + p) * 3 + q) * 2;
    return CMPLX(e[0], e[1]);
}

/* Gauss-Jordan inverse of the sub-block of a 3x3 complex matrix on phases `m`;
 * entries outside the sub-block of the result are 0.  Returns 0 on success. */
static int inv_sub3(const cplx a[3][3], unsigned m, cplx out[3][3]) {
    int idx[3], k = 0;
    for (int p = 0; p < 3; ++p) if (m >> p & 1u) idx[k++] = p;
    cplx w[3][6];
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < 2 * k; ++j)
            w[i][j] = (j < k) ? a[idx[i]][idx[j]] : (j - k == i ? 1.0 : 0.0);
    for (int c = 0; c < k; ++c) {
        int piv = c;
        for (int i = c + 1; i < k; ++i) if (mag(w[i][c]) > mag(w[piv][c])) piv = i;
        if (mag(w[piv][c]) == 0.0) return -1;
        if (piv != c) for (int j = 0; j < 2 * k; ++j) { cplx t = w[c][j]; w[c][j] = w[piv][j]; w[piv][j] = t; }
        cplx d = w[c][c];
        for (int j = 0; j < 2 * k; ++j) w[c][j] /= d;
        for (int i = 0; i < k; ++i) {
            if (i == c) continue;
            cplx f = w[i][c];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * k; ++j) w[i][j] -= f * w[c][j];
        }
    }
    for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q) out[p][q] = 0.0;
    for (int i = 0; i < k; ++i) for (int j = 0; j < k; ++j) out[idx[i]][idx[j]] = w[i][k + j];
    return 0;
}

/* Series admittance of line parent(i) -> i on the phases of bus i. */
static int line_y(const double *z, const unsigned char *ph, int i, cplx y[3][3]) {
    cplx zz[3][3];
    for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q) zz[p][q] = zat(z, i, p, q);
    return inv_sub3(zz, ph[i], y);
}

/* ------------------------------------------------------------------------ */
/* Phase-node numbering: bus order, then phase a,b,c.  idx[bus*3+p] = -1 when
 * phase p is absent.  Returns the number of phase nodes. */
int orc_phase_index(int n, const unsigned char *ph, int *idx) {
    int k = 0;
    for (int i = 0; i < n; ++i)
        for (int p = 0; p < 3; ++p) idx[i * 3 + p] = (ph[i] >> p & 1u) ? k++ : -1;
    return k;
}

/* Dense compact admittance matrix over all phase nodes (root included).
 * Y[r*nphi + c].  Sec. II-A: block Y_ij couples the phases of buses i and j;
 * absent phases are removed (the compact n_phi x n_phi form of the footnote).
 * For a series line with admittance y between p and i: Y_ii += y, Y_pp += y,
 * Y_pi = Y_ip = -y on the phases of i.  Returns 0, or -1 if a line impedance
 * block is singular. */
int orc_ybus(int n, const int *parent, const unsigned char *ph, const double *z,
             double *Yout /* complex [nphi][nphi] */) {
    int *idx = malloc(sizeof(int) * 3 * (size_t)n);
    int nphi = orc_phase_index(n, ph, idx);
    cplx *Y = (cplx *)Yout;
    memset(Y, 0, sizeof(cplx) * (size_t)nphi * nphi);
    int rc = 0;
    for (int i = 1; i < n; ++i) {
        cplx y[3][3];
        if (line_y(z, ph, i, y)) { rc = -1; break; }
        int pb = parent[i];
        for (int p = 0; p < 3; ++p) {
            if (!(ph[i] >> p & 1u)) continue;
            for (int q = 0; q < 3; ++q) {
                if (!(ph[i] >> q & 1u)) continue;
                int ii = idx[i * 3 + p], ij = idx[i * 3 + q];
                int pi = idx[pb * 3 + p], pj = idx[pb * 3 + q];
                Y[(size_t)ii * nphi + ij] += y[p][q];
                Y[(size_t)pi * nphi + pj] += y[p][q];
                Y[(size_t)ii * nphi + pj] -= y[p][q];
                Y[(size_t)pi * nphi + ij] -= y[p][q];
            }
        }
    }
    free(idx);
    return rc;
}

/* Current injection I = Y V computed line by line: the current on line
 * parent(i) -> i is J_i = y_i (V_parent - V_i) on the phases of i, and the
 * injection at a bus is what leaves it through its lines:
 * I_b = sum_{children c} J_c - J_b.  v, iout: [L][n][3] complex. */
int orc_injection(int n, const int *parent, const unsigned char *ph, const double *z,
                  int L, const double *vin, double *iout) {
    const cplx *V = (const cplx *)vin;
    cplx *Inj = (cplx *)iout;
    memset(Inj, 0, sizeof(cplx) * (size_t)L * n * 3);
    for (int i = 1; i < n; ++i) {
        cplx y[3][3];
        if (line_y(z, ph, i, y)) return -1;
        int pb = parent[i];
        for (int l = 0; l < L; ++l) {
            const cplx *Vl = V + (size_t)l * n * 3;
            cplx *Il = Inj + (size_t)l * n * 3;
            for (int p = 0; p < 3; ++p) {
                if (!(ph[i] >> p & 1u)) continue;
                cplx J = 0.0;
                for (int q = 0; q < 3; ++q)
                    if (ph[i] >> q & 1u) J += y[p][q] * (Vl[pb * 3 + q] - Vl[i * 3 + q]);
                Il[pb * 3 + p] += J;
                Il[i * 3 + p] -= J;
            }
        }
    }
    return 0;
}

/* Backward/forward-sweep load flow with constant-power wye loads, one
 * scenario at a time.  Load current drawn at (i,p): conj(S/V).  Backward:
 * branch current J_i = load(i) + sum of children's J.  Forward:
 * V_i = V_parent - z_i J_i.  Stops when max |dV| < tol.  Returns the largest
 * number of sweeps used, or -1 if some scenario did not converge. */
int orc_pf(int n, const int *parent, const unsigned char *ph, const double *z,
           int L, const double *s_load, const double *vslack, double tol, int max_iter,
           double *vout /* [L][n][3] complex */) {
    cplx *V = (cplx *)vout;
    cplx *J = malloc(sizeof(cplx) * 3 * (size_t)n);
    int worst = 0;
    for (int l = 0; l < L; ++l) {
        cplx *Vl = V + (size_t)l * n * 3;
        const cplx *S = (const cplx *)s_load + (size_t)l * n * 3;
        for (int i = 0; i < n; ++i)
            for (int p = 0; p < 3; ++p)
                Vl[i * 3 + p] = (ph[i] >> p & 1u) ? CMPLX(vslack[2 * p], vslack[2 * p + 1]) : 0.0;
        int it, done = 0;
        for (it = 1; it <= max_iter; ++it) {
            memset(J, 0, sizeof(cplx) * 3 * (size_t)n);
            for (int i = n - 1; i >= 1; --i) {
                for (int p = 0; p < 3; ++p)
                    if (ph[i] >> p & 1u) J[i * 3 + p] += conj(S[i * 3 + p] / Vl[i * 3 + p]);
                for (int p = 0; p < 3; ++p) J[parent[i] * 3 + p] += J[i * 3 + p];
            }
            double dmax = 0.0;
            for (int i = 1; i < n; ++i) {
                for (int p = 0; p < 3; ++p) {
                    if (!(ph[i] >> p & 1u)) continue;
                    cplx drop = 0.0;
                    for (int q = 0; q < 3; ++q)
                        if (ph[i] >> q & 1u) drop += zat(z, i, p, q) * J[i * 3 + q];
                    cplx vn = Vl[parent[i] * 3 + p] - drop;
                    double d = mag(vn - Vl[i * 3 + p]);
                    if (!(d <= dmax)) dmax = d;        /* a NaN keeps the sweep from converging */
                    Vl[i * 3 + p] = vn;
                }
            }
            if (dmax < tol) { done = 1; break; }
        }
        if (!done) { free(J); return -1; }
        if (it > worst) worst = it;
    }
    free(J);
    return worst;
}

/* ------------------------------------------------------------------------ */
/* Gaussian elimination of the non-slack rows of Y, one bus (all its phases) at
 * a time, children before parents (i = n-1 ... 1).  In a radial network this
 * order creates no fill: eliminating bus i only changes the diagonal block of
 * its parent, D_p -= Y_pi D_i^{-1} Y_ip = y_i D_i^{-1} y_i.  Stored per bus:
 * yl[i] (line admittance) and Dinv[i] = D_i^{-1}, both 3x3 on the phases of i. */
typedef struct { int n; const int *parent; const unsigned char *ph; cplx (*yl)[3][3]; cplx (*Dinv)[3][3]; } tree_lu;

static int tree_factor(tree_lu *f, int n, const int *parent, const unsigned char *ph, const double *z) {
    f->n = n; f->parent = parent; f->ph = ph;
    f->yl = calloc((size_t)n, sizeof(cplx[3][3]));
    f->Dinv = calloc((size_t)n, sizeof(cplx[3][3]));
    cplx (*D)[3][3] = calloc((size_t)n, sizeof(cplx[3][3]));
    for (int i = 1; i < n; ++i) {
        if (line_y(z, ph, i, f->yl[i])) { free(D); return -1; }
        int pb = parent[i];
        for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q) {
            D[i][p][q] += f->yl[i][p][q];
            if (pb >= 1) D[pb][p][q] += f->yl[i][p][q];
        }
    }
    for (int i = n - 1; i >= 1; --i) {
        if (inv_sub3((const cplx (*)[3])D[i], ph[i], f->Dinv[i])) { free(D); return -1; }
        int pb = parent[i];
        if (pb >= 1) {
            cplx t[3][3] = {{0}}, u[3][3] = {{0}};
            for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q)
                for (int k = 0; k < 3; ++k) t[p][q] += f->yl[i][p][k] * f->Dinv[i][k][q];
            for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q)
                for (int k = 0; k < 3; ++k) u[p][q] += t[p][k] * f->yl[i][k][q];
            for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q) D[pb][p][q] -= u[p][q];
        }
    }
    free(D);
    return 0;
}

static void tree_free(tree_lu *f) { free(f->yl); free(f->Dinv); }

/* Solve Y_LL V_L = b_L - Y_L0 V_0 with the factors: the candidate voltage solve of
 * Algorithm 1 with the slack voltage fixed.  b and V: [n][3]; b[0] is ignored and V[0] is
 * set to v0.  `work` holds n*3 complex numbers. */
static void tree_solve(const tree_lu *f, const cplx *b, const cplx *v0, cplx *V, cplx *work) {
    int n = f->n;
    memcpy(work, b, sizeof(cplx) * 3 * (size_t)n);
    for (int i = n - 1; i >= 1; --i) {            /* forward elimination on b */
        int pb = f->parent[i];
        if (pb < 1) continue;
        cplx t[3] = {0, 0, 0};
        for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q) t[p] += f->Dinv[i][p][q] * work[i * 3 + q];
        for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q) work[pb * 3 + p] += f->yl[i][p][q] * t[q];
    }
    for (int p = 0; p < 3; ++p) V[p] = (f->ph[0] >> p & 1u) ? v0[p] : 0.0;
    for (int i = 1; i < n; ++i) {                 /* back substitution */
        int pb = f->parent[i];
        cplx r[3];
        for (int p = 0; p < 3; ++p) {
            r[p] = work[i * 3 + p];
            for (int q = 0; q < 3; ++q) r[p] += f->yl[i][p][q] * V[pb * 3 + q];
        }
        for (int p = 0; p < 3; ++p) {
            cplx s = 0.0;
            for (int q = 0; q < 3; ++q) s += f->Dinv[i][p][q] * r[q];
            V[i * 3 + p] = (f->ph[i] >> p & 1u) ? s : 0.0;
        }
    }
}

/* Exposed for tests: V = solution of Y_LL V_L = b_L - Y_L0 v0 for L right-hand sides. */
int orc_tree_solve(int n, const int *parent, const unsigned char *ph, const double *z,
                   int L, const double *b, const double *v0, double *vout) {
    tree_lu f;
    if (tree_factor(&f, n, parent, ph, z)) { tree_free(&f); return -1; }
    cplx *work = malloc(sizeof(cplx) * 3 * (size_t)n);
    for (int l = 0; l < L; ++l)
        tree_solve(&f, (const cplx *)b + (size_t)l * n * 3, (const cplx *)v0,
                   (cplx *)vout + (size_t)l * n * 3, work);
    free(work);
    tree_free(&f);
    return 0;
}

/* Z = Y_LL^{-1} over the non-slack phase nodes, column by column: column (j,q)
 * is the solution for a unit injection at (j,q) with V_0 = 0.  Z is stored
 * padded, column-major: Zp[((j*3+q) * n + i) * 3 + p] (zero for the root and
 * for absent phases). */
static int zbus_padded(int n, const int *parent, const unsigned char *ph, const double *z, cplx *Zp) {
    tree_lu f;
    if (tree_factor(&f, n, parent, ph, z)) { tree_free(&f); return -1; }
    memset(Zp, 0, sizeof(cplx) * (size_t)9 * n * n);
    #pragma omp parallel
    {
        cplx *b = calloc(3 * (size_t)n, sizeof(cplx));
        cplx *work = malloc(sizeof(cplx) * 3 * (size_t)n);
        cplx zero3[3] = {0, 0, 0};
        #pragma omp for schedule(static)
        for (int j = 1; j < n; ++j) {
            for (int q = 0; q < 3; ++q) {
                if (!(ph[j] >> q & 1u)) continue;
                memset(b, 0, sizeof(cplx) * 3 * (size_t)n);
                b[j * 3 + q] = 1.0;
                tree_solve(&f, b, zero3, Zp + (size_t)(j * 3 + q) * n * 3, work);
                Zp[(size_t)(j * 3 + q) * n * 3 + 0] = 0.0;
                Zp[(size_t)(j * 3 + q) * n * 3 + 1] = 0.0;
                Zp[(size_t)(j * 3 + q) * n * 3 + 2] = 0.0;
            }
        }
        free(b); free(work);
    }
    tree_free(&f);
    return 0;
}

/* Exposed for tests: the padded Z as above ([3n][n][3] complex). */
int orc_zbus(int n, const int *parent, const unsigned char *ph, const double *z, double *zout) {
    return zbus_padded(n, parent, ph, z, (cplx *)zout);
}

/* ------------------------------------------------------------------------ */
/* Y_Kron (Sec. II-B): Schur complement of Y onto the kept buses.  Each
 * reduced bus is eliminated with all its phases at once (node-level Kron
 * reduction); by the quotient property of Schur complements, eliminating the
 * reduced buses one after another gives Y_KK - Y_KR Y_RR^{-1} Y_RK.  The
 * elimination of bus r updates every pair of buses a, b coupled to r:
 * Y_ab -= Y_ar Y_rr^{-1} Y_rb.  kept[n] is 0/1 (bus 0 must be kept).  Output:
 * Yk[kphi][kphi] over the kept phase nodes in bus/phase order, and kidx[kphi]
 * = bus*3+phase.  Returns kphi, or -1 on a singular block. */
int orc_kron(int n, const int *parent, const unsigned char *ph, const double *z,
             const unsigned char *kept, double *ykout, int *kidx) {
    int *idx = malloc(sizeof(int) * 3 * (size_t)n);
    int nphi = orc_phase_index(n, ph, idx);
    cplx *Y = malloc(sizeof(cplx) * (size_t)nphi * nphi);
    if (orc_ybus(n, parent, ph, z, (double *)Y)) { free(idx); free(Y); return -1; }
    unsigned char *alive = malloc((size_t)n);
    for (int i = 0; i < n; ++i) alive[i] = 1;
    int *nb = malloc(sizeof(int) * (size_t)n);
    for (int r = n - 1; r >= 0; --r) {
        if (kept[r]) continue;
        /* Y_rr^{-1} on the phases of r */
        cplx Yrr[3][3] = {{0}}, Yri[3][3];
        for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q)
            if ((ph[r] >> p & 1u) && (ph[r] >> q & 1u))
                Yrr[p][q] = Y[(size_t)idx[r * 3 + p] * nphi + idx[r * 3 + q]];
        if (inv_sub3((const cplx (*)[3])Yrr, ph[r], Yri)) { free(idx); free(Y); free(alive); free(nb); return -1; }
        /* buses still coupled to r */
        int m = 0;
        for (int a = 0; a < n; ++a) {
            if (!alive[a] || a == r) continue;
            int nz = 0;
            for (int p = 0; p < 3 && !nz; ++p) for (int q = 0; q < 3 && !nz; ++q)
                if ((ph[a] >> p & 1u) && (ph[r] >> q & 1u) && Y[(size_t)idx[a * 3 + p] * nphi + idx[r * 3 + q]] != 0.0) nz = 1;
            if (nz) nb[m++] = a;
        }
        for (int ia = 0; ia < m; ++ia) {
            int a = nb[ia];
            for (int p = 0; p < 3; ++p) {
                if (!(ph[a] >> p & 1u)) continue;
                /* t = Y_a,r(p,:) * Yrr^{-1} */
                cplx t[3] = {0, 0, 0};
                for (int k = 0; k < 3; ++k) {
                    if (!(ph[r] >> k & 1u)) continue;
                    for (int q = 0; q < 3; ++q)
                        if (ph[r] >> q & 1u) t[q] += Y[(size_t)idx[a * 3 + p] * nphi + idx[r * 3 + k]] * Yri[k][q];
                }
                for (int ib = 0; ib < m; ++ib) {
                    int b = nb[ib];
                    for (int q2 = 0; q2 < 3; ++q2) {
                        if (!(ph[b] >> q2 & 1u)) continue;
                        cplx s = 0.0;
                        for (int q = 0; q < 3; ++q)
                            if (ph[r] >> q & 1u) s += t[q] * Y[(size_t)idx[r * 3 + q] * nphi + idx[b * 3 + q2]];
                        Y[(size_t)idx[a * 3 + p] * nphi + idx[b * 3 + q2]] -= s;
                    }
                }
            }
        }
        alive[r] = 0;
    }
    int kphi = 0;
    for (int i = 0; i < n; ++i) if (kept[i]) for (int p = 0; p < 3; ++p) if (ph[i] >> p & 1u) kidx[kphi++] = i * 3 + p;
    cplx *Yk = (cplx *)ykout;
    for (int a = 0; a < kphi; ++a)
        for (int b = 0; b < kphi; ++b)
            Yk[(size_t)a * kphi + b] = Y[(size_t)idx[kidx[a]] * nphi + idx[kidx[b]]];
    free(idx); free(Y); free(alive); free(nb);
    return kphi;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Sec. IV).  Inputs: the feeder (Y through the line impedances),
 * the scenario library vhat/ihat [L][n][3] with Y vhat = ihat, the margin
 * Ebar, the phases.  Additional stop: `max_merges` committed merges (the
 * target reduction).  objective 0 = SMICE (Alg. 1), 1 = max error (eq.
 * iter_obj).  mode 0 = literal (one full solve per candidate), 1 = delta. */
typedef struct {
    int32_t n_iter;          /* merges committed */
    int32_t stop_reason;     /* 0 target reached, 1 no feasible candidate, <0 error */
    int64_t candidates;      /* candidates evaluated over the run */
} orc_summary;

static void aggregate(int n, int L, const int *sup, const cplx *ihat, cplx *Iagg) {
    /* I = (A (x) I_3) Ihat: a super-node carries the sum of its cluster's
     * injections (eq. i_agg); members carry zero. */
    memset(Iagg, 0, sizeof(cplx) * (size_t)L * n * 3);
    for (int l = 0; l < L; ++l)
        for (int i = 0; i < n; ++i)
            for (int p = 0; p < 3; ++p)
                Iagg[((size_t)l * n + sup[i]) * 3 + p] += ihat[((size_t)l * n + i) * 3 + p];
}

/* Delta mode's network solve.  Y Vhat = Ihat holds for the scenario library,
 * so by linearity the solution for injections I is V = Vhat + Y_LL^{-1}(I - Ihat)
 * on the non-slack rows (the slack voltage is the same in both).  This is the
 * same solve as the literal one; written this way its rounding error scales with
 * |I - Ihat| instead of |I|. */
static void solve_from_vhat(const tree_lu *f, int n, int L, const cplx *vhat, const cplx *ihat,
                            const cplx *Iagg, cplx *V, cplx *D, cplx *work) {
    cplx zero3[3] = {0, 0, 0};
    for (size_t k = 0; k < (size_t)L * n * 3; ++k) D[k] = Iagg[k] - ihat[k];
    for (int l = 0; l < L; ++l) {
        tree_solve(f, D + (size_t)l * n * 3, zero3, V + (size_t)l * n * 3, work);
        for (size_t k = 0; k < (size_t)n * 3; ++k) V[(size_t)l * n * 3 + k] += vhat[(size_t)l * n * 3 + k];
    }
}

int orc_reduce(int n, const int *parent, const unsigned char *ph, const double *z,
               int L, const double *vhat_in, const double *ihat_in, const double *vslack,
               double Ebar, int max_merges, int objective, double tau, int mode,
               int record_iters,
               /* outputs */
               int32_t *dec_s, int32_t *dec_r, double *dec_score, double *dec_maxerr,
               double *dec_gap, int32_t *dec_ncand,
               int32_t *super_of, double *vred_out,
               int32_t *rec_s, int32_t *rec_r, double *rec_score, int32_t *rec_count,
               orc_summary *summary) {
    const cplx *vhat = (const cplx *)vhat_in;
    const cplx *ihat = (const cplx *)ihat_in;
    cplx v0[3];
    for (int p = 0; p < 3; ++p) v0[p] = CMPLX(vslack[2 * p], vslack[2 * p + 1]);
    const size_t NL = (size_t)L * n * 3;

    tree_lu f;
    if (tree_factor(&f, n, parent, ph, z)) { tree_free(&f); summary->stop_reason = -1; return -1; }
    cplx *Zp = NULL;
    if (mode == 1) {
        Zp = malloc(sizeof(cplx) * (size_t)9 * n * n);
        if (!Zp || zbus_padded(n, parent, ph, z, Zp)) { tree_free(&f); free(Zp); summary->stop_reason = -2; return -2; }
    }
    double *amag = malloc(sizeof(double) * NL);              /* |Vhat| */
    for (size_t k = 0; k < NL; ++k) amag[k] = mag(vhat[k]);

    /* Alg. 1 state: assignment set S as super_of[] (S = {(sup(i), i)}), the
     * adjacency Lambda (dense n x n, 0/1), the aggregated current I. */
    int *sup = super_of;
    for (int i = 0; i < n; ++i) sup[i] = i;
    unsigned char *Lam = calloc((size_t)n * n, 1);
    for (int i = 1; i < n; ++i) { Lam[(size_t)i * n + parent[i]] = 1; Lam[(size_t)parent[i] * n + i] = 1; }
    cplx *Iagg = malloc(sizeof(cplx) * NL);
    cplx *Vcur = malloc(sizeof(cplx) * NL);
    cplx *Dl = malloc(sizeof(cplx) * NL);
    cplx *work = malloc(sizeof(cplx) * 3 * (size_t)n);
    int *cs = NULL, *cr = NULL;                                   /* candidate lists */
    int cap = 0;
    double *score = NULL, *cmaxe = NULL;
    int merges = 0, stop = 1;
    int64_t total = 0;

    while (merges < max_merges) {
        aggregate(n, L, sup, ihat, Iagg);
        if (mode == 1) solve_from_vhat(&f, n, L, vhat, ihat, Iagg, Vcur, Dl, work);

        /* Candidate set of Algorithm 1: ordered pairs of adjacent super-nodes with
         * phi(r) a subset of phi(s); r is never the slack bus. */
        int nc = 0;
        for (int s = 0; s < n; ++s) {
            if (sup[s] != s) continue;
            for (int r = 1; r < n; ++r) {
                if (!Lam[(size_t)s * n + r]) continue;
                if ((ph[r] & ph[s]) != ph[r]) continue;
                if (nc >= cap) {
                    cap = cap ? 2 * cap : 1024;
                    cs = realloc(cs, sizeof(int) * cap); cr = realloc(cr, sizeof(int) * cap);
                    score = realloc(score, sizeof(double) * cap); cmaxe = realloc(cmaxe, sizeof(double) * cap);
                }
                cs[nc] = s; cr[nc] = r; ++nc;
            }
        }
        if (nc == 0) { stop = 1; break; }
        total += nc;

        /* Independent evaluation of every candidate (the parallel block of Algorithm 1). */
        #pragma omp parallel
        {
            cplx *Ic = malloc(sizeof(cplx) * NL);
            cplx *Vc = malloc(sizeof(cplx) * NL);
            cplx *wk = malloc(sizeof(cplx) * 3 * (size_t)n);
            double *mice = malloc(sizeof(double) * (size_t)L * n);
            int *sup2 = malloc(sizeof(int) * (size_t)n);
            #pragma omp for schedule(dynamic, 4)
            for (int c = 0; c < nc; ++c) {
                int s = cs[c], r = cr[c];
                if (mode == 0) {
                    /* candidate injections: r's current moves onto s; then a full solve */
                    memcpy(Ic, Iagg, sizeof(cplx) * NL);
                    for (int l = 0; l < L; ++l)
                        for (int p = 0; p < 3; ++p) {
                            Ic[((size_t)l * n + s) * 3 + p] += Ic[((size_t)l * n + r) * 3 + p];
                            Ic[((size_t)l * n + r) * 3 + p] = 0.0;
                        }
                    for (int l = 0; l < L; ++l)
                        tree_solve(&f, Ic + (size_t)l * n * 3, v0, Vc + (size_t)l * n * 3, wk);
                } else {
                    /* same solve by linearity: V^c = V + (Z_{:,s} - Z_{:,r}) I_r */
                    memcpy(Vc, Vcur, sizeof(cplx) * NL);
                    for (int l = 0; l < L; ++l)
                        for (int q = 0; q < 3; ++q) {
                            if (!(ph[r] >> q & 1u)) continue;
                            cplx Ir = Iagg[((size_t)l * n + r) * 3 + q];
                            const cplx *zs = Zp + (size_t)(s * 3 + q) * n * 3;
                            const cplx *zr = Zp + (size_t)(r * 3 + q) * n * 3;
                            cplx *Vl = Vc + (size_t)l * n * 3;
                            for (size_t k = 3; k < (size_t)n * 3; ++k) Vl[k] += (zs[k] - zr[k]) * Ir;
                        }
                }
                /* V^c_r <- V^c_s and every member takes its super-node's voltage
                 * (Algorithm 1): post-merge super-node of each bus. */
                for (int i = 0; i < n; ++i) sup2[i] = (sup[i] == r) ? s : sup[i];
                /* per-phase magnitude error and the margin test (Algorithm 1) */
                double maxe = 0.0;
                for (int k = 0; k < L * n; ++k) mice[k] = 0.0;
                for (int l = 0; l < L; ++l)
                    for (int i = 0; i < n; ++i)
                        for (int p = 0; p < 3; ++p) {
                            if (!(ph[i] >> p & 1u)) continue;
                            double e = fabs(amag[((size_t)l * n + i) * 3 + p] - mag(Vc[((size_t)l * n + sup2[i]) * 3 + p]));
                            if (e > maxe) maxe = e;
                            double *m = &mice[(size_t)l * n + sup2[i]];
                            if (e > *m) *m = e;      /* MICE of cluster k: its largest error */
                        }
                cmaxe[c] = maxe;
                if (!(maxe <= Ebar)) { score[c] = INFINITY; continue; }
                if (objective == 1) { score[c] = maxe; continue; }
                double sm = 0.0;                        /* SMICE: sum over l, then over k */
                for (int l = 0; l < L; ++l)
                    for (int k = 0; k < n; ++k)
                        if (sup2[k] == k) sm += mice[(size_t)l * n + k];
                score[c] = sm;
            }
            free(Ic); free(Vc); free(wk); free(mice); free(sup2);
        }

        if (merges < record_iters) {
            rec_count[merges] = nc;
            for (int c = 0; c < nc && c < 2 * n; ++c) {
                rec_s[(size_t)merges * 2 * n + c] = cs[c];
                rec_r[(size_t)merges * 2 * n + c] = cr[c];
                rec_score[(size_t)merges * 2 * n + c] = score[c];
            }
        }

        /* Argmin of Algorithm 1, with the tie band [m, m + tau] and the smallest
         * (r, s) inside it. */
        double m = INFINITY;
        for (int c = 0; c < nc; ++c) if (score[c] < m) m = score[c];
        if (m == INFINITY) { stop = 1; break; }
        int best = -1;
        double gap = INFINITY;
        for (int c = 0; c < nc; ++c) {
            if (score[c] <= m + tau) {
                if (best < 0 || cr[c] < cr[best] || (cr[c] == cr[best] && cs[c] < cs[best])) best = c;
            } else if (score[c] < INFINITY) {
                double g = score[c] - (m + tau);
                if (g < gap) gap = g;
            }
        }
        int S = cs[best], R = cr[best];
        dec_s[merges] = S; dec_r[merges] = R; dec_score[merges] = score[best];
        dec_maxerr[merges] = cmaxe[best]; dec_gap[merges] = gap; dec_ncand[merges] = nc;

        /* Commit (Algorithm 1): the whole cluster of R joins S. */
        for (int i = 0; i < n; ++i) if (sup[i] == R) sup[i] = S;
        /* Adjacency update, eq. (update_adj), for this merge:
         * row/column R fold into S, R loses its edges, no self loop. */
        for (int k = 0; k < n; ++k) {
            if (Lam[(size_t)R * n + k]) { Lam[(size_t)S * n + k] = 1; Lam[(size_t)k * n + S] = 1; }
            Lam[(size_t)R * n + k] = 0; Lam[(size_t)k * n + R] = 0;
        }
        Lam[(size_t)S * n + S] = 0;
        ++merges;
        stop = 0;
    }
    if (merges >= max_merges) stop = 0;

    /* Reduced-network voltages: I = A Ihat, solve, each bus takes its
     * super-node's voltage. */
    aggregate(n, L, sup, ihat, Iagg);
    cplx *Vf = malloc(sizeof(cplx) * NL);
    if (mode == 1) solve_from_vhat(&f, n, L, vhat, ihat, Iagg, Vf, Dl, work);
    else for (int l = 0; l < L; ++l) tree_solve(&f, Iagg + (size_t)l * n * 3, v0, Vf + (size_t)l * n * 3, work);
    cplx *vred = (cplx *)vred_out;
    for (int l = 0; l < L; ++l)
        for (int i = 0; i < n; ++i)
            for (int p = 0; p < 3; ++p)
                vred[((size_t)l * n + i) * 3 + p] = (ph[i] >> p & 1u) ? Vf[((size_t)l * n + sup[i]) * 3 + p] : 0.0;

    summary->n_iter = merges;
    summary->stop_reason = stop;
    summary->candidates = total;
    free(Vf); free(amag); free(Lam); free(Iagg); free(Vcur); free(Dl); free(work);
    free(cs); free(cr); free(score); free(cmaxe); free(Zp);
    tree_free(&f);
    return 0;
}

void orc_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
