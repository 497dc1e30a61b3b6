/*
 * tc_oracle.c -- plain, slow, FP64 CPU oracle for Tavis-Cummings unitary
 * evolution (arXiv 2403.06937).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or helper with the GPU library, and the GPU library never calls it.
 *
 * Conventions (the paper fixes the model, not the indexing):
 *   n atoms, N = 2^n basis states (Sec. II, Eq. 2: |l_1 ... l_n>).
 *   Basis index s: atom i (1-based) is bit (n - i) of s, so atom 1 is the most
 *   significant bit -- the order of the tensor product in Eq. 2.
 *   l_i(s) = that bit; number of excited atoms = popcount(s).
 *   The system is closed (Sec. II, text after Eq. 1), so the free-photon
 *   number is fixed by the atoms: p(s) = n - popcount(s).  The basis is the
 *   n-excitation manifold, of dimension exactly 2^n.
 *   hbar = 1.
 *   Complex arrays are interleaved (re, im) doubles, row-major.
 *
 * Hamiltonian (Sec. II, Eq. 4, rotating-wave form):
 *   H = w_c a^dag a + sum_i [ w_a sigma_i^dag sigma_i
 *                             + g_i (a^dag sigma_i + a sigma_i^dag) ].
 *   Diagonal:      H_ss = w_c * p(s) + w_a * popcount(s).
 *   Off-diagonal:  s_e has atom i excited and p photons; s_g = s_e with atom i
 *                  relaxed, holding p + 1 photons.  a^dag sigma_i maps s_e to
 *                  s_g with amplitude sqrt(p + 1) (bosonic mode), so
 *                  H[s_g][s_e] = H[s_e][s_g] = g_i * sqrt(p(s_e) + 1).
 *   Coupling switch 1 ("qubit-photon"): the reading of Eq. 1 in which every
 *   atom owns one photon qubit; the element is then g_i, without the
 *   square root.
 *
 * Evolution (Sec. III.A, Eqs. 6-8): rho(t+dt) = e^{-iHdt} rho(t) e^{iHdt}.
 * The Lindblad term of Eq. 5 is switched off, as in the paper.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

static int popcount_u(unsigned long s) {
    int c = 0;
    while (s) { c += (int)(s & 1ul); s >>= 1; }
    return c;
}

/* Coupling element between s_e (atom excited) and s_g (same atom relaxed).
 * Eq. 4: g_i times the photon creation amplitude sqrt(p(s_e)+1). */
static double coupling_element(int n, const double* g, int atom0, unsigned long s_e, int coupling) {
    int p = n - popcount_u(s_e);
    if (coupling == 1) return g[atom0];
    return g[atom0] * sqrt((double)(p + 1));
}

static double diagonal_element(int n, double wa, double wc, unsigned long s) {
    int pc = popcount_u(s);
    int p = n - pc;
    double a = wc * (double)p;
    double b = wa * (double)pc;
    return a + b;
}

/* ---------------------------------------------------------------------- */
/* O-H: dense Hamiltonian (Eq. 4 on the basis of Eq. 2), row-major N x N.   */
void orc_build_h_dense(int n, const double* g, double wa, double wc, int coupling, double* H) {
    unsigned long N = 1ul << n;
    memset(H, 0, sizeof(double) * N * N);
    for (unsigned long s = 0; s < N; s++) {
        H[s * N + s] = diagonal_element(n, wa, wc, s);
        for (int i = 1; i <= n; i++) {
            unsigned long bit = 1ul << (n - i);
            if (s & bit) {                       /* atom i excited in s */
                unsigned long sg = s & ~bit;     /* atom i relaxed: one more photon */
                double h = coupling_element(n, g, i - 1, s, coupling);
                H[sg * N + s] = h;
                H[s * N + sg] = h;
            }
        }
    }
}

/* y = H x for complex x, using the structure of Eq. 4 directly (no matrix). */
static void h_apply(int n, const double* g, double wa, double wc, int coupling,
                    const double* x, double* y) {
    unsigned long N = 1ul << n;
    for (unsigned long s = 0; s < N; s++) {
        double d = diagonal_element(n, wa, wc, s);
        y[2 * s] = d * x[2 * s];
        y[2 * s + 1] = d * x[2 * s + 1];
    }
    for (unsigned long s = 0; s < N; s++) {
        for (int i = 1; i <= n; i++) {
            unsigned long bit = 1ul << (n - i);
            if (!(s & bit)) continue;
            unsigned long sg = s & ~bit;
            double h = coupling_element(n, g, i - 1, s, coupling);
            y[2 * sg] += h * x[2 * s];
            y[2 * sg + 1] += h * x[2 * s + 1];
            y[2 * s] += h * x[2 * sg];
            y[2 * s + 1] += h * x[2 * sg + 1];
        }
    }
}

/* ---------------------------------------------------------------------- */
/* O-psi: one step psi <- exp(-i H dt) psi by the Taylor series of Eq. 7,
 * summed until the newest term is below tol * |psi| (max-norm).  Returns the
 * number of terms used, or -1 if 200 terms did not converge. */
int orc_state_step(int n, const double* g, double wa, double wc, int coupling,
                   double dt, double tol, double* psi) {
    unsigned long N = 1ul << n;
    double* term = (double*)malloc(sizeof(double) * 2 * N);
    double* hx = (double*)malloc(sizeof(double) * 2 * N);
    double* acc = (double*)malloc(sizeof(double) * 2 * N);
    double scale = 0.0;
    for (unsigned long j = 0; j < 2 * N; j++) {
        term[j] = psi[j];
        acc[j] = psi[j];
        if (fabs(psi[j]) > scale) scale = fabs(psi[j]);
    }
    int k, used = -1;
    for (k = 1; k <= 200; k++) {
        /* term_k = (-i dt / k) H term_{k-1} */
        h_apply(n, g, wa, wc, coupling, term, hx);
        double f = dt / (double)k, big = 0.0;
        for (unsigned long j = 0; j < N; j++) {
            double re = hx[2 * j], im = hx[2 * j + 1];
            /* (-i)(re + i im) = im - i re */
            term[2 * j] = f * im;
            term[2 * j + 1] = -f * re;
            acc[2 * j] += term[2 * j];
            acc[2 * j + 1] += term[2 * j + 1];
            if (fabs(term[2 * j]) > big) big = fabs(term[2 * j]);
            if (fabs(term[2 * j + 1]) > big) big = fabs(term[2 * j + 1]);
        }
        if (big <= tol * scale) { used = k; break; }
    }
    memcpy(psi, acc, sizeof(double) * 2 * N);
    free(term); free(hx); free(acc);
    return used;
}

/* ---------------------------------------------------------------------- */
/* Observables of one density matrix (complex N x N), the row layout
 *   [P_1..P_n, <p>, P(0..n), Tr rho, Tr rho^2, E]          (2n+5 values)
 * P_i = sum_s rho_ss l_i(s)       (excited population of atom i)
 * <p>  = sum_s rho_ss p(s)        (mean free-photon number)
 * P(m) = sum_{popcount(s) = n-m} rho_ss: probability of m free photons, the
 *        projector reading of the photon-number states of Eq. 13
 * Tr rho, Tr rho^2 = sum_ij |rho_ij|^2, E = Tr(H rho). */
void orc_observables(int n, const double* g, double wa, double wc, int coupling,
                     const double* rho, double* out) {
    unsigned long N = 1ul << n;
    int stride = 2 * n + 5;
    for (int j = 0; j < stride; j++) out[j] = 0.0;
    double* Pi = out;
    double* pmean = out + n;
    double* Pm = out + n + 1;
    double* tr = out + 2 * n + 2;
    double* pur = out + 2 * n + 3;
    double* en = out + 2 * n + 4;
    for (unsigned long s = 0; s < N; s++) {
        double d = rho[2 * (s * N + s)];
        int pc = popcount_u(s);
        for (int i = 1; i <= n; i++)
            if ((s >> (n - i)) & 1ul) Pi[i - 1] += d;
        *pmean += d * (double)(n - pc);
        Pm[n - pc] += d;
        *tr += d;
        *en += diagonal_element(n, wa, wc, s) * d;
    }
    for (unsigned long a = 0; a < N; a++)
        for (unsigned long b = 0; b < N; b++) {
            double re = rho[2 * (a * N + b)], im = rho[2 * (a * N + b) + 1];
            *pur += re * re + im * im;
        }
    /* off-diagonal part of Tr(H rho) = sum_{a != b} H_ab rho_ba */
    for (unsigned long s = 0; s < N; s++)
        for (int i = 1; i <= n; i++) {
            unsigned long bit = 1ul << (n - i);
            if (!(s & bit)) continue;
            unsigned long sg = s & ~bit;
            double h = coupling_element(n, g, i - 1, s, coupling);
            *en += h * (rho[2 * (s * N + sg)] + rho[2 * (sg * N + s)]);
        }
}

/* The same observables for a pure state rho = psi psi^dag, without forming rho. */
void orc_observables_pure(int n, const double* g, double wa, double wc, int coupling,
                          const double* psi, double* out) {
    unsigned long N = 1ul << n;
    int stride = 2 * n + 5;
    for (int j = 0; j < stride; j++) out[j] = 0.0;
    double nrm = 0.0;
    for (unsigned long s = 0; s < N; s++) {
        double d = psi[2 * s] * psi[2 * s] + psi[2 * s + 1] * psi[2 * s + 1];
        int pc = popcount_u(s);
        for (int i = 1; i <= n; i++)
            if ((s >> (n - i)) & 1ul) out[i - 1] += d;
        out[n] += d * (double)(n - pc);
        out[n + 1 + (n - pc)] += d;
        nrm += d;
    }
    out[2 * n + 2] = nrm;
    out[2 * n + 3] = nrm * nrm;           /* Tr (psi psi^dag)^2 = |psi|^4 */
    double* hx = (double*)malloc(sizeof(double) * 2 * N);
    h_apply(n, g, wa, wc, coupling, psi, hx);
    double e = 0.0;
    for (unsigned long s = 0; s < N; s++)
        e += psi[2 * s] * hx[2 * s] + psi[2 * s + 1] * hx[2 * s + 1];
    out[2 * n + 4] = e;                   /* <psi|H|psi>, real for Hermitian H */
    free(hx);
}

/* ---------------------------------------------------------------------- */
/* O-dense: U = exp(-i H dt), built column by column by stepping e_j with
 * orc_state_step.  U is complex N x N, row-major. */
int orc_expm_columns(int n, const double* g, double wa, double wc, int coupling,
                     double dt, double tol, double* U) {
    unsigned long N = 1ul << n;
    double* col = (double*)malloc(sizeof(double) * 2 * N);
    int worst = 0;
    for (unsigned long j = 0; j < N; j++) {
        memset(col, 0, sizeof(double) * 2 * N);
        col[2 * j] = 1.0;
        int k = orc_state_step(n, g, wa, wc, coupling, dt, tol, col);
        if (k < 0) { worst = -1; }
        else if (worst >= 0 && k > worst) worst = k;
        for (unsigned long i = 0; i < N; i++) {
            U[2 * (i * N + j)] = col[2 * i];
            U[2 * (i * N + j) + 1] = col[2 * i + 1];
        }
    }
    free(col);
    return worst;
}

/* Dense one-step map of Eq. 6, rows [r0, r1) of rho' = U rho U^dag, with plain
 * triple loops: X_i. = sum_k U_ik rho_k.,  rho'_ij = sum_k X_ik conj(U_jk).
 * rho and U are complex N x N; out receives rows r0..r1-1 (row r0 first). */
void orc_dense_step_rows(long N, const double* U, const double* rho, double* out, long r0, long r1) {
    #pragma omp parallel for schedule(dynamic, 1)
    for (long i = r0; i < r1; i++) {
        double* x = (double*)calloc(2 * (size_t)N, sizeof(double));
        for (long k = 0; k < N; k++) {
            double ur = U[2 * (i * N + k)], ui = U[2 * (i * N + k) + 1];
            if (ur == 0.0 && ui == 0.0) continue;
            const double* rk = rho + 2 * k * N;
            for (long j = 0; j < N; j++) {
                double rr = rk[2 * j], ri = rk[2 * j + 1];
                x[2 * j] += ur * rr - ui * ri;
                x[2 * j + 1] += ur * ri + ui * rr;
            }
        }
        double* o = out + 2 * (i - r0) * N;
        for (long j = 0; j < N; j++) {
            const double* uj = U + 2 * j * N;
            double sr = 0.0, si = 0.0;
            for (long k = 0; k < N; k++) {
                double xr = x[2 * k], xi = x[2 * k + 1];
                double ur = uj[2 * k], ui = -uj[2 * k + 1];   /* conj(U_jk) */
                sr += xr * ur - xi * ui;
                si += xr * ui + xi * ur;
            }
            o[2 * j] = sr;
            o[2 * j + 1] = si;
        }
        free(x);
    }
}

/* Plain complex matrix product C = A B (N x N, interleaved), triple loop. */
void orc_zgemm(long N, const double* A, const double* B, double* C) {
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        double* c = C + 2 * i * N;
        for (long j = 0; j < 2 * N; j++) c[j] = 0.0;
        for (long k = 0; k < N; k++) {
            double ar = A[2 * (i * N + k)], ai = A[2 * (i * N + k) + 1];
            const double* b = B + 2 * k * N;
            for (long j = 0; j < N; j++) {
                c[2 * j] += ar * b[2 * j] - ai * b[2 * j + 1];
                c[2 * j + 1] += ar * b[2 * j + 1] + ai * b[2 * j];
            }
        }
    }
}

/* Eq. 10 as printed: L = sum_{k=0}^{kmax} (-i H dt)^k / k!, built from dense
 * products of the full (unshifted, unscaled) matrix, as the paper does with
 * k_max = 10.  H is real N x N; L is complex N x N. */
void orc_taylor_fixed(long N, const double* H, double dt, int kmax, double* L) {
    size_t NN = (size_t)N * (size_t)N;
    double* A = (double*)malloc(sizeof(double) * 2 * NN);
    double* P = (double*)malloc(sizeof(double) * 2 * NN);
    double* T = (double*)malloc(sizeof(double) * 2 * NN);
    for (size_t e = 0; e < NN; e++) {          /* A = -i H dt */
        A[2 * e] = 0.0;
        A[2 * e + 1] = -H[e] * dt;
    }
    memset(P, 0, sizeof(double) * 2 * NN);     /* P = A^0 = I */
    memset(L, 0, sizeof(double) * 2 * NN);
    for (long i = 0; i < N; i++) { P[2 * (i * N + i)] = 1.0; L[2 * (i * N + i)] = 1.0; }
    double fact = 1.0;
    for (int k = 1; k <= kmax; k++) {
        orc_zgemm(N, A, P, T);                 /* P = A^k */
        memcpy(P, T, sizeof(double) * 2 * NN);
        fact *= (double)k;
        for (size_t e = 0; e < 2 * NN; e++) L[e] += P[e] / fact;
    }
    free(A); free(P); free(T);
}

/* ---------------------------------------------------------------------- */
/* O-eig: cyclic Jacobi eigenvalue method for a real symmetric matrix
 * (the textbook two-sided rotation sweep).  A (n x n, row-major) is
 * overwritten; on return w holds eigenvalues and V (row-major) the
 * eigenvectors as columns, A = V diag(w) V^T.  Returns the sweeps used. */
int orc_jacobi_eig(int m, double* A, double* V, double* w) {
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) V[i * m + j] = (i == j) ? 1.0 : 0.0;
    int sweep;
    for (sweep = 0; sweep < 100; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++) {
                tot += A[i * m + j] * A[i * m + j];
                if (i != j) off += A[i * m + j] * A[i * m + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < m - 1; p++)
            for (int q = p + 1; q < m; q++) {
                double apq = A[p * m + q];
                if (apq == 0.0) continue;
                double app = A[p * m + p], aqq = A[q * m + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; k++) {        /* A <- A J (columns p, q) */
                    double akp = A[k * m + p], akq = A[k * m + q];
                    A[k * m + p] = c * akp - s * akq;
                    A[k * m + q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; k++) {        /* A <- J^T A (rows p, q) */
                    double apk = A[p * m + k], aqk = A[q * m + k];
                    A[p * m + k] = c * apk - s * aqk;
                    A[q * m + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; k++) {        /* V <- V J */
                    double vkp = V[k * m + p], vkq = V[k * m + q];
                    V[k * m + p] = c * vkp - s * vkq;
                    V[k * m + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < m; i++) w[i] = A[i * m + i];
    return sweep;
}

/* O-Dicke: the (n+1) x (n+1) tridiagonal of Eq. 4 with all g_i = g, on the
 * symmetric states |m> = (n - m excited atoms, symmetrised) x (m photons).
 * D_mm = w_c m + w_a (n - m);  D_{m,m+1} = g (m+1) sqrt(n - m), from
 * a^dag J_- with J_- |j, m_z> = sqrt((j + m_z)(j - m_z + 1)) |j, m_z - 1>,
 * j = n/2, m_z = (n - m) - n/2. */
void orc_dicke_matrix(int n, double g, double wa, double wc, double* D) {
    int m1 = n + 1;
    for (int a = 0; a < m1 * m1; a++) D[a] = 0.0;
    for (int m = 0; m <= n; m++) {
        D[m * m1 + m] = wc * (double)m + wa * (double)(n - m);
        if (m < n) {
            double h = g * (double)(m + 1) * sqrt((double)(n - m));
            D[m * m1 + m + 1] = h;
            D[(m + 1) * m1 + m] = h;
        }
    }
}

/* ---------------------------------------------------------------------- */
/* O-grad (forward mode).  For one parameter theta with dH = dH/dtheta, the
 * pair (dpsi, psi) obeys i d/dt [dpsi; psi] = [[H, dH], [0, H]] [dpsi; psi],
 * so one step is the exponential of the block upper-triangular generator
 * (Van Loan's identity: its upper-right block is the Frechet derivative of
 * exp).  It is applied here by its Taylor series until the newest term is
 * below tol.  param: 0..n-1 -> g_{param+1}; n -> w_a; n+1 -> w_c. */
static void dh_apply(int n, const double* g, int coupling, int param,
                     const double* x, double* y) {
    unsigned long N = 1ul << n;
    for (unsigned long j = 0; j < 2 * N; j++) y[j] = 0.0;
    if (param == n || param == n + 1) {
        for (unsigned long s = 0; s < N; s++) {
            int pc = popcount_u(s);
            double d = (param == n) ? (double)pc : (double)(n - pc);
            y[2 * s] = d * x[2 * s];
            y[2 * s + 1] = d * x[2 * s + 1];
        }
        return;
    }
    double* unit = (double*)calloc((size_t)n, sizeof(double));
    unit[param] = 1.0;
    (void)g;
    unsigned long bit = 1ul << (n - 1 - param);
    for (unsigned long s = 0; s < N; s++) {
        if (!(s & bit)) continue;
        unsigned long sg = s & ~bit;
        double h = coupling_element(n, unit, param, s, coupling);
        y[2 * sg] += h * x[2 * s];
        y[2 * sg + 1] += h * x[2 * s + 1];
        y[2 * s] += h * x[2 * sg];
        y[2 * s + 1] += h * x[2 * sg + 1];
    }
    free(unit);
}

int orc_tangent_step(int n, const double* g, double wa, double wc, int coupling, int param,
                     double dt, double tol, double* dpsi, double* psi) {
    unsigned long N = 1ul << n;
    size_t sz = sizeof(double) * 2 * N;
    double *tu = (double*)malloc(sz), *tv = (double*)malloc(sz);
    double *au = (double*)malloc(sz), *av = (double*)malloc(sz);
    double *h1 = (double*)malloc(sz), *h2 = (double*)malloc(sz), *h3 = (double*)malloc(sz);
    memcpy(tu, dpsi, sz); memcpy(au, dpsi, sz);
    memcpy(tv, psi, sz);  memcpy(av, psi, sz);
    double scale = 0.0;
    for (unsigned long j = 0; j < 2 * N; j++) {
        if (fabs(psi[j]) > scale) scale = fabs(psi[j]);
        if (fabs(dpsi[j]) > scale) scale = fabs(dpsi[j]);
    }
    int used = -1;
    for (int k = 1; k <= 200; k++) {
        /* [u; v] <- (-i dt / k) [H u + dH v; H v] */
        h_apply(n, g, wa, wc, coupling, tu, h1);
        dh_apply(n, g, coupling, param, tv, h2);
        h_apply(n, g, wa, wc, coupling, tv, h3);
        double f = dt / (double)k, big = 0.0;
        for (unsigned long j = 0; j < N; j++) {
            double ur = h1[2 * j] + h2[2 * j], ui = h1[2 * j + 1] + h2[2 * j + 1];
            double vr = h3[2 * j], vi = h3[2 * j + 1];
            tu[2 * j] = f * ui;  tu[2 * j + 1] = -f * ur;
            tv[2 * j] = f * vi;  tv[2 * j + 1] = -f * vr;
            au[2 * j] += tu[2 * j]; au[2 * j + 1] += tu[2 * j + 1];
            av[2 * j] += tv[2 * j]; av[2 * j + 1] += tv[2 * j + 1];
            double m1 = fabs(tu[2 * j]) > fabs(tu[2 * j + 1]) ? fabs(tu[2 * j]) : fabs(tu[2 * j + 1]);
            double m2 = fabs(tv[2 * j]) > fabs(tv[2 * j + 1]) ? fabs(tv[2 * j]) : fabs(tv[2 * j + 1]);
            if (m1 > big) big = m1;
            if (m2 > big) big = m2;
        }
        if (big <= tol * scale) { used = k; break; }
    }
    memcpy(dpsi, au, sz); memcpy(psi, av, sz);
    free(tu); free(tv); free(au); free(av); free(h1); free(h2); free(h3);
    return used;
}
