/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle for the lattice Boltzmann
 * collide-and-stream update of Latt, Coreixas & Beny, "Cross-platform
 * programming model for many-core lattice Boltzmann simulation"
 * (arXiv:2010.11751).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker that the CUDA library
 * is compared against.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or generator with the CUDA library: velocity sets, weights, the
 * moment basis and its inverse are all built here, from their definitions.
 *
 * What it computes (one time iteration, Section 2.1, Eqs. of the collision
 * and streaming steps):
 *   1. for every fluid cell x:  f_out(x) = Omega(f(x))
 *   2. for every direction k:   if x + c_k is fluid, f_k(x + c_k) <- f_out_k(x)
 *                               else  f_kbar(x) <- f_out_k(x) - 6 t_k rho_w c_k.u_w
 *      (link-wise bounce-back with momentum exchange, Section 2.1, rho_w = 1)
 *   into a fresh array, with periodic wrap at the domain faces.  orc_step_curved
 *   places walls at a fraction of their links (the curved-wall extension of
 *   link-wise bounce-back the paper points to in Section 1; see there).
 * Solid cells hold zeros.  Every scheme and layout of the paper computes this
 * same map (end of Section 2.3), so the oracle implements only this plain
 * two-array form.
 *
 * Collision models (Section 2.2, Section 2.6).  The paper gives the framework
 * (raw moments, their relaxation, the bulk-viscosity coupling and one worked
 * inversion example) but points to an external appendix for the full model
 * formulas.  The readings used here are:
 *   BGK_W2  second-order weighted equilibrium; the printed |u|^2 coefficient is
 *           read as the standard -3/2 |u|^2 (the only value that conserves mass
 *           and keeps the opposite-direction symmetry of Section 2.6 valid).
 *   BGK_NW4 BGK towards the non-weighted equilibrium: f_eq = T^-1 M_eq with the
 *           product-Maxwellian raw moments m0 = 1, m1 = u, m2 = u^2 + cs^2.
 *   TRT     symmetric / antisymmetric parts relaxed with w+ = omega and w-
 *           from the magic parameter Lambda = (1/w+ - 1/2)(1/w- - 1/2).
 *   REG     regularized: f_out = E + (1-omega) t_k/(2 cs^4) H2_k : Pi_neq.
 *   RR      recursive regularized in Hermite-moment form: second-order
 *           non-equilibrium Hermite moments relaxed (with bulk coupling), every
 *           higher basis moment rebuilt as equilibrium + the recursive product
 *           of velocities and post-collision second-order non-equilibrium.
 *   RM, HM, CM, CHM, K
 *           moments in raw, Hermite, central, central-Hermite or cumulant space
 *           over the lattice's monomial basis, relaxed as in the raw-moment
 *           relaxation equation of Section 2.6; second-order diagonal moments
 *           use the bulk-viscosity coupling of Section 2.6 (with the reading
 *           M*_200 = M_200 - w+(M_200 - Meq_200) - w-(M_020 - Meq_020)
 *                         - w-(M_002 - Meq_002), cyclically);
 *           off-diagonal second order relaxes with omega; order >= 3 with
 *           omega_high.  Post-collision moments go back to raw moments and
 *           f_out = T^-1 (rho M*), which is the route of Section 2.6.
 *
 * Lattices: D3Q19 (the paper's) and D3Q27.  Velocity ordering: the vectors
 * whose first non-zero component is -1, sorted by |c|^2 then
 * lexicographically (-1 < 0 < 1), then the rest vector, then the negated
 * first half.  This gives c_0 = (-1,0,0) = -c_10 for D3Q19 (Section 2.6).
 *
 * Pins (tests/test_oracle_*.py, against what the mathematics fixes, not
 * against this file): worked inversion example and equilibrium symmetry of
 * Section 2.6; exact mass and momentum conservation; equilibrium as a fixed
 * point; omega = 1 gives the equilibrium; each model's per-moment relaxation
 * law recomputed independently; reductions of RM, HM, CM, CHM to BGK_NW4 at
 * equal rates; cumulants against log-moment-generating-function derivatives;
 * Couette and TRT Poiseuille exactness, Taylor-Green decay and its order of
 * convergence; hand-enumerated pulls on tiny lattices; traversal-order
 * independence; walls at a fraction of their links (orc_step_curved): the
 * halfway case equal to the plain step bit for bit, Couette flow between
 * off-lattice walls exact, Poiseuille flow second-order convergent.  No
 * function here is parity unpinned.
 *
 * Compile with -ffp-contract=off so that each operation rounds once.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXQ 27
#define CS2 (1.0 / 3.0)

enum { M_BGK_W2 = 0, M_BGK_NW4, M_TRT, M_REG, M_RR, M_RM, M_HM, M_CM, M_CHM, M_K, M_COUNT };

typedef struct {
    int Q;
    int c[ORC_MAXQ][3];
    double t[ORC_MAXQ];
    int opp[ORC_MAXQ];
    int rest;
    int pqr[ORC_MAXQ][3];      /* monomial basis c_x^p c_y^q c_z^r */
    int T[ORC_MAXQ][ORC_MAXQ]; /* T[j][k] = monomial j evaluated at c_k */
    double Tinv[ORC_MAXQ][ORC_MAXQ];
    int ready;
} lat_t;

static lat_t g_lat19, g_lat27;

/* ------------------------------------------------------------------ */
/* exact rational arithmetic for the moment-matrix inverse             */
/* ------------------------------------------------------------------ */
typedef struct { int64_t n, d; } frac_t;

static int64_t gcd64(int64_t a, int64_t b) {
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b) { int64_t r = a % b; a = b; b = r; }
    return a ? a : 1;
}
static frac_t fr_make(int64_t n, int64_t d) {
    if (d < 0) { n = -n; d = -d; }
    int64_t g = gcd64(n, d);
    frac_t r = { n / g, d / g };
    return r;
}
static frac_t fr_sub(frac_t a, frac_t b) { return fr_make(a.n * b.d - b.n * a.d, a.d * b.d); }
static frac_t fr_mul(frac_t a, frac_t b) { return fr_make(a.n * b.n, a.d * b.d); }
static frac_t fr_div(frac_t a, frac_t b) { return fr_make(a.n * b.d, a.d * b.n); }

/* Gauss-Jordan elimination with row pivoting, in exact fractions. */
static int invert_exact(int n, int A[ORC_MAXQ][ORC_MAXQ], double out[ORC_MAXQ][ORC_MAXQ]) {
    static frac_t M[ORC_MAXQ][2 * ORC_MAXQ];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j)
            M[i][j] = fr_make(j < n ? A[i][j] : (j - n == i ? 1 : 0), 1);
    for (int col = 0; col < n; ++col) {
        int piv = -1;
        for (int r = col; r < n; ++r)
            if (M[r][col].n != 0) { piv = r; break; }
        if (piv < 0) return -1; /* singular */
        if (piv != col)
            for (int j = 0; j < 2 * n; ++j) { frac_t tmp = M[col][j]; M[col][j] = M[piv][j]; M[piv][j] = tmp; }
        frac_t p = M[col][col];
        for (int j = 0; j < 2 * n; ++j) M[col][j] = fr_div(M[col][j], p);
        for (int r = 0; r < n; ++r) {
            if (r == col || M[r][col].n == 0) continue;
            frac_t fct = M[r][col];
            for (int j = 0; j < 2 * n; ++j) M[r][j] = fr_sub(M[r][j], fr_mul(fct, M[col][j]));
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) out[i][j] = (double)M[i][n + j].n / (double)M[i][n + j].d;
    return 0;
}

/* ------------------------------------------------------------------ */
/* lattice construction                                                */
/* ------------------------------------------------------------------ */
static int ipow(int b, int e) { int r = 1; while (e-- > 0) r *= b; return r; }

static int build_lattice(lat_t* L, int Q) {
    int half[13][3], nh = 0;
    /* nested loops visit {-1,0,1}^3 in lexicographic order (-1 < 0 < 1) */
    for (int norm = 1; norm <= 3; ++norm)
        for (int a = -1; a <= 1; ++a)
            for (int b = -1; b <= 1; ++b)
                for (int c = -1; c <= 1; ++c) {
                    int n2 = a * a + b * b + c * c;
                    if (n2 != norm) continue;
                    if (Q == 19 && n2 > 2) continue;
                    int first = a != 0 ? a : (b != 0 ? b : c);
                    if (first != -1) continue;
                    half[nh][0] = a; half[nh][1] = b; half[nh][2] = c; ++nh;
                }
    if (2 * nh + 1 != Q) return -1;
    L->Q = Q;
    L->rest = nh;
    for (int k = 0; k < nh; ++k)
        for (int d = 0; d < 3; ++d) {
            L->c[k][d] = half[k][d];
            L->c[k + nh + 1][d] = -half[k][d];
        }
    for (int d = 0; d < 3; ++d) L->c[nh][d] = 0;
    for (int k = 0; k < Q; ++k) {
        int n2 = L->c[k][0] * L->c[k][0] + L->c[k][1] * L->c[k][1] + L->c[k][2] * L->c[k][2];
        if (Q == 19) L->t[k] = n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        else L->t[k] = n2 == 0 ? 8.0 / 27.0 : (n2 == 1 ? 2.0 / 27.0 : (n2 == 2 ? 1.0 / 54.0 : 1.0 / 216.0));
        for (int m = 0; m < Q; ++m)
            if (L->c[m][0] == -L->c[k][0] && L->c[m][1] == -L->c[k][1] && L->c[m][2] == -L->c[k][2]) L->opp[k] = m;
    }
    /* monomial basis */
    static const int b19[19][3] = {
        {0,0,0}, {1,0,0},{0,1,0},{0,0,1},
        {2,0,0},{0,2,0},{0,0,2},{1,1,0},{1,0,1},{0,1,1},
        {1,2,0},{1,0,2},{2,1,0},{0,1,2},{2,0,1},{0,2,1},
        {2,2,0},{2,0,2},{0,2,2}};
    static const int b27[27][3] = {
        {0,0,0}, {1,0,0},{0,1,0},{0,0,1},
        {2,0,0},{0,2,0},{0,0,2},{1,1,0},{1,0,1},{0,1,1},
        {1,2,0},{1,0,2},{2,1,0},{0,1,2},{2,0,1},{0,2,1},{1,1,1},
        {2,2,0},{2,0,2},{0,2,2},{2,1,1},{1,2,1},{1,1,2},
        {2,2,1},{2,1,2},{1,2,2},
        {2,2,2}};
    for (int j = 0; j < Q; ++j)
        for (int d = 0; d < 3; ++d) L->pqr[j][d] = Q == 19 ? b19[j][d] : b27[j][d];
    for (int j = 0; j < Q; ++j)
        for (int k = 0; k < Q; ++k)
            L->T[j][k] = ipow(L->c[k][0], L->pqr[j][0]) * ipow(L->c[k][1], L->pqr[j][1]) *
                         ipow(L->c[k][2], L->pqr[j][2]);
    if (invert_exact(Q, L->T, L->Tinv) != 0) return -2;
    L->ready = 1;
    return 0;
}

static const lat_t* get_lat(int Q) {
    lat_t* L = Q == 19 ? &g_lat19 : (Q == 27 ? &g_lat27 : NULL);
    if (!L) return NULL;
    if (!L->ready) {
#ifdef _OPENMP
#pragma omp critical(orc_lattice_init)
#endif
        {
            if (!L->ready) build_lattice(L, Q);
        }
    }
    return L->ready ? L : NULL;
}

static int basis_index(const lat_t* L, int p, int q, int r) {
    for (int j = 0; j < L->Q; ++j)
        if (L->pqr[j][0] == p && L->pqr[j][1] == q && L->pqr[j][2] == r) return j;
    return -1;
}

/* ------------------------------------------------------------------ */
/* moments                                                             */
/* ------------------------------------------------------------------ */
/* one-dimensional polynomial families: monomial xi^p or Hermite h_p(xi) */
static double poly1(int hermite, int p, double xi) {
    if (p == 0) return 1.0;
    if (p == 1) return xi;
    /* p == 2 */
    return hermite ? xi * xi - CS2 : xi * xi;
}

/* X_j = sum_k phi_j(c_k - shift) f_k / rho  for every basis element j */
static void moments_generic(const lat_t* L, int hermite, const double shift[3], const double* f, double rho,
                            double* X) {
    for (int j = 0; j < L->Q; ++j) {
        double s = 0.0;
        for (int k = 0; k < L->Q; ++k) {
            double v = 1.0;
            for (int d = 0; d < 3; ++d) v *= poly1(hermite, L->pqr[j][d], (double)L->c[k][d] - shift[d]);
            s += v * f[k];
        }
        X[j] = s / rho;
    }
}

/* Hermite (central or not) -> monomial (central or not): xi^2 = h2 + cs^2 h0 */
static void hermite_to_monomial(const lat_t* L, const double* a, double* M) {
    static const double E[3][3] = {{1, 0, 0}, {0, 1, 0}, {CS2, 0, 1}};
    for (int j = 0; j < L->Q; ++j) {
        int p = L->pqr[j][0], q = L->pqr[j][1], r = L->pqr[j][2];
        double s = 0.0;
        for (int a0 = 0; a0 <= p; ++a0)
            for (int b0 = 0; b0 <= q; ++b0)
                for (int c0 = 0; c0 <= r; ++c0) {
                    double e = E[p][a0] * E[q][b0] * E[r][c0];
                    if (e == 0.0) continue;
                    s += e * a[basis_index(L, a0, b0, c0)];
                }
        M[j] = s;
    }
}

/* central monomial moments -> raw monomial moments: c^p = sum_a C(p,a) u^(p-a) xi^a */
static void central_to_raw(const lat_t* L, const double u[3], const double* kappa, double* M) {
    static const int C[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}};
    for (int j = 0; j < L->Q; ++j) {
        int p = L->pqr[j][0], q = L->pqr[j][1], r = L->pqr[j][2];
        double s = 0.0;
        for (int a0 = 0; a0 <= p; ++a0)
            for (int b0 = 0; b0 <= q; ++b0)
                for (int c0 = 0; c0 <= r; ++c0) {
                    double coef = (double)(C[p][a0] * C[q][b0] * C[r][c0]);
                    double up = 1.0;
                    for (int e = 0; e < p - a0; ++e) up *= u[0];
                    for (int e = 0; e < q - b0; ++e) up *= u[1];
                    for (int e = 0; e < r - c0; ++e) up *= u[2];
                    s += coef * up * kappa[basis_index(L, a0, b0, c0)];
                }
        M[j] = s;
    }
}

/* f = T^-1 (rho * Mhat) */
static void populations_from_raw(const lat_t* L, double rho, const double* Mhat, double* f) {
    for (int k = 0; k < L->Q; ++k) {
        double s = 0.0;
        for (int j = 0; j < L->Q; ++j) s += L->Tinv[k][j] * (rho * Mhat[j]);
        f[k] = s;
    }
}

static void density_velocity(const lat_t* L, const double* f, double* rho, double u[3]) {
    double r = 0.0, j[3] = {0, 0, 0};
    for (int k = 0; k < L->Q; ++k) {
        r += f[k];
        for (int d = 0; d < 3; ++d) j[d] += (double)L->c[k][d] * f[k];
    }
    *rho = r;
    for (int d = 0; d < 3; ++d) u[d] = j[d] / r;
}

/* ------------------------------------------------------------------ */
/* equilibria                                                          */
/* ------------------------------------------------------------------ */
static void eq_w2(const lat_t* L, double rho, const double u[3], double* E) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int k = 0; k < L->Q; ++k) {
        double cu = L->c[k][0] * u[0] + L->c[k][1] * u[1] + L->c[k][2] * u[2];
        E[k] = rho * L->t[k] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

static double maxwell1(int p, double u) { return p == 0 ? 1.0 : (p == 1 ? u : u * u + CS2); }

static void eq_raw_moments(const lat_t* L, const double u[3], double* Meq) {
    for (int j = 0; j < L->Q; ++j)
        Meq[j] = maxwell1(L->pqr[j][0], u[0]) * maxwell1(L->pqr[j][1], u[1]) * maxwell1(L->pqr[j][2], u[2]);
}

static void eq_nw4(const lat_t* L, double rho, const double u[3], double* E) {
    double Meq[ORC_MAXQ];
    eq_raw_moments(L, u, Meq);
    populations_from_raw(L, rho, Meq, E);
}

/* ------------------------------------------------------------------ */
/* relaxation in a moment space                                        */
/* ------------------------------------------------------------------ */
typedef struct { double omega, omega_bulk, omega_high, lambda; } prm_t;

static int order_of(const lat_t* L, int j) { return L->pqr[j][0] + L->pqr[j][1] + L->pqr[j][2]; }
static int is_diag2(const lat_t* L, int j) {
    return order_of(L, j) == 2 && (L->pqr[j][0] == 2 || L->pqr[j][1] == 2 || L->pqr[j][2] == 2);
}

/* X* for every basis element: conserved orders keep their equilibrium value,
 * second order uses omega (off-diagonal) or the bulk coupling (diagonal),
 * orders >= 3 use omega_high. */
static void relax(const lat_t* L, const prm_t* P, const double* X, const double* Xeq, double* Xs) {
    double wm = (P->omega_bulk - P->omega) / 3.0;
    double wp = wm + P->omega;
    int d2[3] = {basis_index(L, 2, 0, 0), basis_index(L, 0, 2, 0), basis_index(L, 0, 0, 2)};
    for (int j = 0; j < L->Q; ++j) {
        int o = order_of(L, j);
        if (o <= 1) Xs[j] = Xeq[j];
        else if (o == 2 && !is_diag2(L, j)) Xs[j] = X[j] - P->omega * (X[j] - Xeq[j]);
        else if (o == 2) {
            double s = X[j];
            for (int a = 0; a < 3; ++a) {
                double w = d2[a] == j ? wp : wm;
                s -= w * (X[d2[a]] - Xeq[d2[a]]);
            }
            Xs[j] = s;
        } else Xs[j] = X[j] - P->omega_high * (X[j] - Xeq[j]);
    }
}

/* ------------------------------------------------------------------ */
/* cumulants: moment-cumulant relation over set partitions              */
/* ------------------------------------------------------------------ */
/* For a basis element of order n, the positions 0..n-1 carry the axes
 * (x repeated p times, y q times, z r times).  The central moment of the
 * element equals the sum, over all set partitions of the positions into
 * blocks of size >= 2 (first central moments vanish), of the product of the
 * cumulants of the blocks. */
#define MAXPART 256
#define MAXBLK 3
typedef struct {
    int nparts;
    int nblocks[MAXPART];
    int block[MAXPART][MAXBLK]; /* basis index of each block */
} partlist_t;

static partlist_t g_parts19[19], g_parts27[27];
static int g_parts_ready19, g_parts_ready27;

static void build_partitions(const lat_t* L, partlist_t* PL) {
    for (int j = 0; j < L->Q; ++j) {
        int axes[6], n = 0;
        for (int d = 0; d < 3; ++d)
            for (int e = 0; e < L->pqr[j][d]; ++e) axes[n++] = d;
        partlist_t* P = &PL[j];
        P->nparts = 0;
        if (n < 2) continue;
        /* restricted growth strings a[0..n-1], a[0]=0, a[i] <= 1+max(a[0..i-1]) */
        int a[6] = {0};
        for (;;) {
            int nb = 0;
            for (int i = 0; i < n; ++i) if (a[i] + 1 > nb) nb = a[i] + 1;
            int cnt[6][3] = {{0}}, sz[6] = {0}, ok = 1;
            for (int i = 0; i < n; ++i) { cnt[a[i]][axes[i]]++; sz[a[i]]++; }
            for (int b = 0; b < nb; ++b) if (sz[b] < 2) ok = 0;
            if (ok && nb <= MAXBLK) {
                int idx = P->nparts++;
                P->nblocks[idx] = nb;
                for (int b = 0; b < nb; ++b) P->block[idx][b] = basis_index(L, cnt[b][0], cnt[b][1], cnt[b][2]);
            }
            /* next restricted growth string */
            int i = n - 1;
            for (; i >= 1; --i) {
                int mx = 0;
                for (int m = 0; m < i; ++m) if (a[m] > mx) mx = a[m];
                if (a[i] <= mx) { a[i]++; for (int m = i + 1; m < n; ++m) a[m] = 0; break; }
            }
            if (i < 1) break;
        }
    }
}

static const partlist_t* get_parts(const lat_t* L) {
    partlist_t* PL = L->Q == 19 ? g_parts19 : g_parts27;
    int* ready = L->Q == 19 ? &g_parts_ready19 : &g_parts_ready27;
    if (!*ready) {
#ifdef _OPENMP
#pragma omp critical(orc_parts_init)
#endif
        {
            if (!*ready) { build_partitions(L, PL); *ready = 1; }
        }
    }
    return PL;
}

/* basis is ordered by increasing total order, so lower-order cumulants are
 * always available when an element is processed */
static void central_to_cumulant(const lat_t* L, const double* kappa, double* K) {
    const partlist_t* PL = get_parts(L);
    for (int j = 0; j < L->Q; ++j) {
        int o = order_of(L, j);
        if (o == 0) { K[j] = 1.0; continue; }
        if (o == 1) { K[j] = 0.0; continue; }
        double s = kappa[j];
        for (int p = 0; p < PL[j].nparts; ++p) {
            if (PL[j].nblocks[p] == 1) continue; /* the element itself */
            double prod = 1.0;
            for (int b = 0; b < PL[j].nblocks[p]; ++b) prod *= K[PL[j].block[p][b]];
            s -= prod;
        }
        K[j] = s;
    }
}

static void cumulant_to_central(const lat_t* L, const double* K, double* kappa) {
    const partlist_t* PL = get_parts(L);
    for (int j = 0; j < L->Q; ++j) {
        int o = order_of(L, j);
        if (o == 0) { kappa[j] = 1.0; continue; }
        if (o == 1) { kappa[j] = 0.0; continue; }
        double s = 0.0;
        for (int p = 0; p < PL[j].nparts; ++p) {
            double prod = 1.0;
            for (int b = 0; b < PL[j].nblocks[p]; ++b) prod *= K[PL[j].block[p][b]];
            s += prod;
        }
        kappa[j] = s;
    }
}

/* ------------------------------------------------------------------ */
/* collision operators                                                 */
/* ------------------------------------------------------------------ */
static void collide(const lat_t* L, int model, const prm_t* P, const double* f, double* fout) {
    const int Q = L->Q;
    double rho, u[3];
    density_velocity(L, f, &rho, u);
    const double zero[3] = {0, 0, 0};
    double X[ORC_MAXQ] = {0}, Xeq[ORC_MAXQ] = {0}, Xs[ORC_MAXQ] = {0}, Ms[ORC_MAXQ] = {0}, tmp[ORC_MAXQ] = {0},
           E[ORC_MAXQ] = {0};

    switch (model) {
    case M_BGK_W2:
        eq_w2(L, rho, u, E);
        for (int k = 0; k < Q; ++k) fout[k] = f[k] - P->omega * (f[k] - E[k]);
        return;
    case M_BGK_NW4:
        eq_nw4(L, rho, u, E);
        for (int k = 0; k < Q; ++k) fout[k] = f[k] - P->omega * (f[k] - E[k]);
        return;
    case M_TRT: {
        double wp = P->omega;
        double wmi = 0.5 + P->lambda / (1.0 / wp - 0.5);
        double wm = 1.0 / wmi;
        eq_w2(L, rho, u, E);
        for (int k = 0; k < Q; ++k) {
            int kb = L->opp[k];
            double fp = 0.5 * (f[k] + f[kb]), fm = 0.5 * (f[k] - f[kb]);
            double ep = 0.5 * (E[k] + E[kb]), em = 0.5 * (E[k] - E[kb]);
            fout[k] = f[k] - wp * (fp - ep) - wm * (fm - em);
        }
        return;
    }
    case M_REG: {
        eq_w2(L, rho, u, E);
        double Pi[3][3] = {{0}};
        for (int k = 0; k < Q; ++k)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Pi[a][b] += (double)(L->c[k][a] * L->c[k][b]) * (f[k] - E[k]);
        for (int k = 0; k < Q; ++k) {
            double hp = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    hp += ((double)(L->c[k][a] * L->c[k][b]) - (a == b ? CS2 : 0.0)) * Pi[a][b];
            fout[k] = E[k] + (1.0 - P->omega) * L->t[k] / (2.0 * CS2 * CS2) * hp;
        }
        return;
    }
    case M_RR: {
        moments_generic(L, 1, zero, f, rho, X);
        for (int j = 0; j < Q; ++j) {
            Xeq[j] = 1.0;
            for (int d = 0; d < 3; ++d)
                for (int e = 0; e < L->pqr[j][d]; ++e) Xeq[j] *= u[d];
        }
        /* second order: relax (the relax() rule for orders <= 2) */
        relax(L, P, X, Xeq, Xs);
        double neq2[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                int p[3] = {0, 0, 0};
                p[a]++; p[b]++;
                int j = basis_index(L, p[0], p[1], p[2]);
                neq2[a][b] = Xs[j] - Xeq[j];
            }
        for (int j = 0; j < Q; ++j) {
            int o = order_of(L, j);
            if (o < 3) continue;
            int axes[6], n = 0;
            for (int d = 0; d < 3; ++d)
                for (int e = 0; e < L->pqr[j][d]; ++e) axes[n++] = d;
            double s = 0.0;
            for (int i1 = 0; i1 < n; ++i1)
                for (int i2 = i1 + 1; i2 < n; ++i2) {
                    double prod = neq2[axes[i1]][axes[i2]];
                    for (int l = 0; l < n; ++l)
                        if (l != i1 && l != i2) prod *= u[axes[l]];
                    s += prod;
                }
            Xs[j] = Xeq[j] + s;
        }
        hermite_to_monomial(L, Xs, Ms);
        populations_from_raw(L, rho, Ms, fout);
        return;
    }
    case M_RM:
        moments_generic(L, 0, zero, f, rho, X);
        eq_raw_moments(L, u, Xeq);
        relax(L, P, X, Xeq, Ms);
        populations_from_raw(L, rho, Ms, fout);
        return;
    case M_HM:
        moments_generic(L, 1, zero, f, rho, X);
        for (int j = 0; j < Q; ++j) {
            Xeq[j] = 1.0;
            for (int d = 0; d < 3; ++d)
                for (int e = 0; e < L->pqr[j][d]; ++e) Xeq[j] *= u[d];
        }
        relax(L, P, X, Xeq, Xs);
        hermite_to_monomial(L, Xs, Ms);
        populations_from_raw(L, rho, Ms, fout);
        return;
    case M_CM:
        moments_generic(L, 0, u, f, rho, X);
        for (int j = 0; j < Q; ++j)
            Xeq[j] = maxwell1(L->pqr[j][0], 0.0) * maxwell1(L->pqr[j][1], 0.0) * maxwell1(L->pqr[j][2], 0.0);
        relax(L, P, X, Xeq, Xs);
        central_to_raw(L, u, Xs, Ms);
        populations_from_raw(L, rho, Ms, fout);
        return;
    case M_CHM:
        moments_generic(L, 1, u, f, rho, X);
        for (int j = 0; j < Q; ++j) Xeq[j] = j == 0 ? 1.0 : 0.0;
        relax(L, P, X, Xeq, Xs);
        hermite_to_monomial(L, Xs, tmp);
        central_to_raw(L, u, tmp, Ms);
        populations_from_raw(L, rho, Ms, fout);
        return;
    case M_K:
        moments_generic(L, 0, u, f, rho, tmp);
        central_to_cumulant(L, tmp, X);
        for (int j = 0; j < Q; ++j) Xeq[j] = (j == 0) ? 1.0 : (is_diag2(L, j) ? CS2 : 0.0);
        relax(L, P, X, Xeq, Xs);
        cumulant_to_central(L, Xs, tmp);
        central_to_raw(L, u, tmp, Ms);
        populations_from_raw(L, rho, Ms, fout);
        return;
    default:
        for (int k = 0; k < Q; ++k) fout[k] = f[k];
    }
}

/* ------------------------------------------------------------------ */
/* exported API                                                        */
/* ------------------------------------------------------------------ */
#define EXPORT __attribute__((visibility("default")))

static prm_t make_prm(const double* params) {
    prm_t P = {params[0], params[1], params[2], params[3]};
    return P;
}

/* velocity set: c[Q*3], t[Q], opp[Q]; returns Q or <0 */
EXPORT int orc_lattice(int Q, int* c, double* t, int* opp) {
    const lat_t* L = get_lat(Q);
    if (!L) return -1;
    for (int k = 0; k < Q; ++k) {
        for (int d = 0; d < 3; ++d) c[3 * k + d] = L->c[k][d];
        t[k] = L->t[k];
        opp[k] = L->opp[k];
    }
    return Q;
}

/* monomial basis exponents pqr[Q*3] and the exact inverse Tinv[Q*Q] (row k = population) */
EXPORT int orc_moment_basis(int Q, int* pqr, double* Tinv) {
    const lat_t* L = get_lat(Q);
    if (!L) return -1;
    for (int j = 0; j < Q; ++j)
        for (int d = 0; d < 3; ++d) pqr[3 * j + d] = L->pqr[j][d];
    for (int k = 0; k < Q; ++k)
        for (int j = 0; j < Q; ++j) Tinv[k * Q + j] = L->Tinv[k][j];
    return 0;
}

/* kind 0: second-order weighted (BGK_W2/TRT/REG); kind 1: non-weighted product Maxwellian */
EXPORT int orc_equilibrium(int Q, int kind, double rho, const double* u, double* feq) {
    const lat_t* L = get_lat(Q);
    if (!L) return -1;
    if (kind == 0) eq_w2(L, rho, u, feq);
    else eq_nw4(L, rho, u, feq);
    return 0;
}

/* the equilibrium that a collision model relaxes towards */
EXPORT int orc_model_equilibrium(int Q, int model, double rho, const double* u, double* feq) {
    int kind = (model == M_BGK_W2 || model == M_TRT || model == M_REG) ? 0 : 1;
    return orc_equilibrium(Q, kind, rho, u, feq);
}

/* params = {omega, omega_bulk, omega_high, trt_lambda} */
EXPORT int orc_collide(int Q, int model, const double* params, const double* f, double* fout) {
    const lat_t* L = get_lat(Q);
    if (!L || model < 0 || model >= M_COUNT) return -1;
    prm_t P = make_prm(params);
    collide(L, model, &P, f, fout);
    return 0;
}

/* per-unit-mass cumulants over the basis (order 0 reported as 1, order 1 as 0) */
EXPORT int orc_cumulants(int Q, const double* f, double* K) {
    const lat_t* L = get_lat(Q);
    if (!L) return -1;
    double rho, u[3], kap[ORC_MAXQ];
    density_velocity(L, f, &rho, u);
    moments_generic(L, 0, u, f, rho, kap);
    central_to_cumulant(L, kap, K);
    return 0;
}

static inline int64_t wrapi(int64_t a, int64_t n) { a %= n; return a < 0 ? a + n : a; }

/* One time iteration of the plain two-array definition.
 * f, fnew: SoA [Q][N], N = nx*ny*nz, cell index i = (x*ny + y)*nz + z.
 * flags[N]: 0 fluid, 1 resting wall, 2..7 moving wall (velocity wall_u[3*flag]).
 * force: NULL or a constant acceleration g, added after collision as
 *        3 t_k c_k.g (test hook for body-force driven flows; not part of the
 *        paper's method).
 * perm: NULL (natural order) or a permutation of 0..N-1 giving the traversal
 *       order; nthreads > 1 parallelises the natural-order traversal. */
static int step_impl(int Q, int nx, int ny, int nz, const uint8_t* flags, const double* wall_u, int model,
                     const double* params, const double* force, const int64_t* perm, int nthreads,
                     const double* qfrac, const double* f, double* fnew);

EXPORT int orc_step(int Q, int nx, int ny, int nz, const uint8_t* flags, const double* wall_u, int model,
                    const double* params, const double* force, const int64_t* perm, int nthreads,
                    const double* f, double* fnew) {
    return step_impl(Q, nx, ny, nz, flags, wall_u, model, params, force, perm, nthreads, NULL, f, fnew);
}

/* The same iteration with walls at a fraction of their links (the extension to
 * curved boundaries the paper points to in Section 1: link-wise and entirely
 * local).  qfrac [Q][N]: for a fluid cell x and a link k whose neighbour x + c_k
 * is solid, q = qfrac[k*N + i] in (0, 1] is the fraction of the link from x at
 * which the wall lies; other entries are ignored.  The reflected population is
 * the linear interpolation of Bouzidi, Firdaouss & Lallemand (2001), with
 * W = -6 t_k rho_w c_k.u_w:
 *   q >= 1/2:  f_kbar(x, t+1) = [f_out_k(x) + W] / (2q) + (2q - 1)/(2q) f_out_kbar(x)
 *   q <  1/2:  f_kbar(x, t+1) = 2q f_out_k(x) + (1 - 2q) f_k(x, t) + W
 * In the second form, f_k(x, t) -- the population that streamed into x from
 * x - c_k -- stands for that neighbour's post-collision f_out_k(x - c_k), so that
 * the rule stays local to x (it is the same value one step earlier, and equal to
 * it in a steady flow).  q = 1/2 gives the halfway bounce-back exactly.  force:
 * as in orc_step. */
EXPORT int orc_step_curved(int Q, int nx, int ny, int nz, const uint8_t* flags, const double* wall_u, int model,
                           const double* params, const double* force, const double* qfrac, int nthreads,
                           const double* f, double* fnew) {
    return step_impl(Q, nx, ny, nz, flags, wall_u, model, params, force, NULL, nthreads, qfrac, f, fnew);
}

static int step_impl(int Q, int nx, int ny, int nz, const uint8_t* flags, const double* wall_u, int model,
                     const double* params, const double* force, const int64_t* perm, int nthreads,
                     const double* qfrac, const double* f, double* fnew) {
    const lat_t* L = get_lat(Q);
    if (!L || nx < 1 || ny < 1 || nz < 1 || model < 0 || model >= M_COUNT) return -1;
    if (model == M_RR || model == M_K) get_parts(L);
    const int64_t N = (int64_t)nx * ny * nz;
    prm_t P = make_prm(params);
    memset(fnew, 0, sizeof(double) * (size_t)Q * (size_t)N);
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1) if (perm == NULL && nthreads > 1)
#endif
    for (int64_t it = 0; it < N; ++it) {
        int64_t i = perm ? perm[it] : it;
        if (flags[i] != 0) continue;
        int x = (int)(i / ((int64_t)ny * nz));
        int y = (int)((i / nz) % ny);
        int z = (int)(i % nz);
        double fc[ORC_MAXQ], fo[ORC_MAXQ];
        for (int k = 0; k < Q; ++k) fc[k] = f[(int64_t)k * N + i];
        collide(L, model, &P, fc, fo);
        if (force)
            for (int k = 0; k < Q; ++k)
                fo[k] += 3.0 * L->t[k] * (L->c[k][0] * force[0] + L->c[k][1] * force[1] + L->c[k][2] * force[2]);
        for (int k = 0; k < Q; ++k) {
            int64_t xn = wrapi(x + L->c[k][0], nx), yn = wrapi(y + L->c[k][1], ny), zn = wrapi(z + L->c[k][2], nz);
            int64_t j = (xn * ny + yn) * nz + zn;
            int fl = flags[j];
            if (fl == 0) {
                fnew[(int64_t)k * N + j] = fo[k];
            } else {
                const double* uw = wall_u + 3 * fl;
                double cu = L->c[k][0] * uw[0] + L->c[k][1] * uw[1] + L->c[k][2] * uw[2];
                double W = -6.0 * L->t[k] * 1.0 * cu;
                double v = fo[k] + W;
                if (qfrac) {
                    double q = qfrac[(int64_t)k * N + i];
                    if (q >= 0.5)
                        v = (fo[k] + W) / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * fo[L->opp[k]];
                    else
                        v = 2.0 * q * fo[k] + (1.0 - 2.0 * q) * fc[k] + W;
                }
                fnew[(int64_t)L->opp[k] * N + i] = v;
            }
        }
    }
    return 0;
}

/* nsteps iterations in place on f (scratch of the same size allocated here) */
EXPORT int orc_run(int Q, int nx, int ny, int nz, const uint8_t* flags, const double* wall_u, int model,
                   const double* params, const double* force, int nsteps, int nthreads, double* f) {
    const int64_t N = (int64_t)nx * ny * nz;
    double* tmp = (double*)malloc(sizeof(double) * (size_t)Q * (size_t)N);
    if (!tmp) return -2;
    int rc = 0;
    for (int s = 0; s < nsteps && rc == 0; ++s) {
        rc = orc_step(Q, nx, ny, nz, flags, wall_u, model, params, force, NULL, nthreads, f, tmp);
        memcpy(f, tmp, sizeof(double) * (size_t)Q * (size_t)N);
    }
    free(tmp);
    return rc;
}

/* rho[N], u[3][N] (SoA); solid cells report rho = 1 and the wall velocity */
EXPORT int orc_macroscopic(int Q, int64_t N, const uint8_t* flags, const double* wall_u, const double* f,
                           double* rho, double* u) {
    const lat_t* L = get_lat(Q);
    if (!L) return -1;
    for (int64_t i = 0; i < N; ++i) {
        if (flags[i] != 0) {
            rho[i] = 1.0;
            for (int d = 0; d < 3; ++d) u[d * N + i] = wall_u[3 * flags[i] + d];
            continue;
        }
        double fc[ORC_MAXQ], r, uu[3];
        for (int k = 0; k < Q; ++k) fc[k] = f[(int64_t)k * N + i];
        density_velocity(L, fc, &r, uu);
        rho[i] = r;
        for (int d = 0; d < 3; ++d) u[d * N + i] = uu[d];
    }
    return 0;
}

/* mass = sum rho, energy = sum rho |u|^2 / 2, over fluid cells */
EXPORT int orc_conserved(int Q, int64_t N, const uint8_t* flags, const double* f, double* mass, double* energy) {
    const lat_t* L = get_lat(Q);
    if (!L) return -1;
    double m = 0.0, e = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        if (flags[i] != 0) continue;
        double fc[ORC_MAXQ], r, uu[3];
        for (int k = 0; k < Q; ++k) fc[k] = f[(int64_t)k * N + i];
        density_velocity(L, fc, &r, uu);
        m += r;
        e += 0.5 * r * (uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
    }
    *mass = m;
    *energy = e;
    return 0;
}

/* f = the model's own equilibrium of rho[N], u[3][N] on every fluid cell
 * (rho or u may be NULL: rho = 1, u = 0); solid cells get 0.  A whole-field
 * loop of orc_model_equilibrium, for initialising large lattices. */
EXPORT int orc_init_equilibrium_field(int Q, int model, int64_t N, const uint8_t* flags, const double* rho,
                                      const double* u, double* f) {
    const lat_t* L = get_lat(Q);
    if (!L) return -1;
    for (int64_t i = 0; i < N; ++i) {
        double fe[ORC_MAXQ] = {0};
        if (flags[i] == 0) {
            double uu[3] = {u ? u[i] : 0.0, u ? u[N + i] : 0.0, u ? u[2 * N + i] : 0.0};
            if (orc_model_equilibrium(Q, model, rho ? rho[i] : 1.0, uu, fe) != 0) return -1;
        }
        for (int k = 0; k < Q; ++k) f[(int64_t)k * N + i] = fe[k];
    }
    return 0;
}
