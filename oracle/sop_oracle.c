/*
 * sop_oracle.c -- plain FP64 CPU oracle for the Fourier split-operator (FSO)
 * time step of Bauke & Keitel, "Accelerating the Fourier split operator
 * method via graphics processing units" (arXiv:1012.3911).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load this library.  The GPU
 * library never links it, calls it or shares code, headers or tables with it.
 *
 * It is the method written out plainly, in the paper's order and notation:
 *   - its own mixed radix-2/3 FFT (Sec. 2.1: on a lattice the continuous
 *     Fourier transform becomes a DFT) and an O(n^2) DFT by definition that
 *     the tests use to pin the FFT;
 *   - one Strang step  U_A1(1/2) F^-1 U~_A2(1) F U_A1(1/2)  (Eqs. 6-8), for
 *     the Schroedinger split (Eqs. 10a/10b, actions Eqs. 11 and 13) and the
 *     Dirac split (Eqs. 18a/18b); the two half steps of a step use the same
 *     interval integral with delta = 1/2 and adjacent half steps are NOT
 *     merged;
 *   - the Dirac real-space factor from the exp-alpha identity (Eqs. 23, 26)
 *     and the Dirac kinetic factor u(p)^dagger diag(...) u(p) with u(p)
 *     built literally from d_+-, beta and alpha_i (Eqs. 29, 30, 33);
 *   - norm and field-free energy with compensated (Kahan) sums.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   lattice  x_{a,j} = -n_a h_a / 2 + j h_a, j = 0..n_a-1, periodic;
 *   momenta  p_{a,k} = hbar 2 pi kappa_k / (n_a h_a), kappa_k = k for
 *            2k < n_a else k - n_a (the Nyquist index of an even side maps
 *            to -n_a/2);
 *   forward  X_k = sum_j x_j exp(-2 pi i jk/n) (the sign of Eq. 12);
 *   inverse  x_j = (1/n) sum_k X_k exp(+2 pi i jk/n);
 *   the time integrals of Eqs. 11, 13 and 25a use the midpoint rule: the
 *   caller passes the field at t_n + tau/2, held constant over the step;
 *   Schroedinger length gauge: q phi = V - q x.E (V is the potential energy);
 *   Dirac: the uniform vector potential enters the real-space factor.
 *
 * Layout: arrays are C-ordered with axis 0 (x) fastest: psi[c][z][y][x],
 * interleaved complex double.  dims[0] = n_x.
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

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------ */
/* Threads                                                             */
/* ------------------------------------------------------------------ */

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }

int orc_get_threads(void) { return g_threads; }

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Discrete Fourier transform                                          */
/* ------------------------------------------------------------------ */

/* 1 if n = 2^a 3^b with n >= 1 (the sizes the radix-2/3 FFT handles). */
int orc_size_ok(int64_t n) {
    if (n < 1) return 0;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

/* DFT by its definition, O(n^2): out[k] = sum_j in[j] exp(sign 2 pi i jk/n).
 * The product jk is reduced mod n in integers so the angle stays exact. */
void orc_dft_naive(const cplx *in, cplx *out, int64_t n, int sign) {
    for (int64_t k = 0; k < n; ++k) {
        cplx acc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            int64_t e = (j * k) % n;
            double ang = sign * TWO_PI * (double)e / (double)n;
            acc += in[j] * (cos(ang) + I * sin(ang));
        }
        out[k] = acc;
    }
}

/* Table w[e] = exp(sign 2 pi i e / N), e = 0..N-1. */
static cplx *make_roots(int64_t N, int sign) {
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    for (int64_t e = 0; e < N; ++e) {
        double ang = sign * TWO_PI * (double)e / (double)N;
        w[e] = cos(ang) + I * sin(ang);
    }
    return w;
}

/* Recursive decimation-in-time Cooley-Tukey for n = 2^a 3^b.
 * out[k] = sum_{j<n} in[j*istride] W_n^{jk}, with W_n^e = w[e * wstep] and
 * w the root table of the top-level size (n * wstep = N).
 * Split by the radix r (2 while n is even, else 3): the r decimated
 * subsequences in[(r j' + q) istride] give sub-DFTs Y_q of size m = n/r, and
 *   X[k + m s] = sum_q W_n^{q (k + m s)} Y_q[k],  s = 0..r-1.              */
static void fft_rec(const cplx *in, int64_t istride, cplx *out, int64_t n,
                    const cplx *w, int64_t wstep) {
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    const int r = (n % 2 == 0) ? 2 : 3;
    const int64_t m = n / r;
    for (int q = 0; q < r; ++q)
        fft_rec(in + q * istride, istride * r, out + q * m, m, w, wstep * r);
    for (int64_t k = 0; k < m; ++k) {
        cplx y[3];
        for (int q = 0; q < r; ++q) y[q] = out[q * m + k];
        for (int s = 0; s < r; ++s) {
            cplx acc = 0.0;
            for (int q = 0; q < r; ++q) {
                int64_t e = ((int64_t)q * (k + m * s)) % n;
                acc += w[e * wstep] * y[q];
            }
            out[k + m * s] = acc;
        }
    }
}

/* In-place 1D FFT of x[0..n-1]; sign -1 forward, +1 inverse (unscaled). */
int orc_fft(cplx *x, int64_t n, int sign) {
    if (!orc_size_ok(n)) return -1;
    cplx *w = make_roots(n, sign);
    cplx *a = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    memcpy(a, x, sizeof(cplx) * (size_t)n);
    fft_rec(a, 1, x, n, w, 1);
    free(a);
    free(w);
    return 0;
}

/* FFT along one axis of a C-ordered array with dims[0] fastest, applied to
 * every pencil; unscaled. */
static void fft_axis(cplx *data, int ndim, const int64_t *dims, int axis, int sign) {
    int64_t n = dims[axis];
    int64_t inner = 1, outer = 1;
    for (int a = 0; a < axis; ++a) inner *= dims[a];
    for (int a = axis + 1; a < ndim; ++a) outer *= dims[a];
    const int64_t npencil = inner * outer;
    cplx *w = make_roots(n, sign);
#pragma omp parallel num_threads(g_threads)
    {
        cplx *a = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *b = (cplx *)malloc(sizeof(cplx) * (size_t)n);
#pragma omp for schedule(static)
        for (int64_t p = 0; p < npencil; ++p) {
            int64_t o = p / inner, i = p % inner;
            cplx *base = data + o * inner * n + i;
            for (int64_t j = 0; j < n; ++j) a[j] = base[j * inner];
            fft_rec(a, 1, b, n, w, 1);
            for (int64_t j = 0; j < n; ++j) base[j * inner] = b[j];
        }
        free(a);
        free(b);
    }
    free(w);
}

/* d-dimensional DFT (separable, Sec. 2.1).  sign -1: forward, unscaled.
 * sign +1: inverse including the 1/N factor. */
int orc_fftn(cplx *data, int ndim, const int64_t *dims, int sign) {
    int64_t N = 1;
    for (int a = 0; a < ndim; ++a) {
        if (!orc_size_ok(dims[a])) return -1;
        N *= dims[a];
    }
    for (int a = 0; a < ndim; ++a) fft_axis(data, ndim, dims, a, sign);
    if (sign > 0) {
        const double s = 1.0 / (double)N;
#pragma omp parallel for num_threads(g_threads) schedule(static)
        for (int64_t j = 0; j < N; ++j) data[j] *= s;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Lattices                                                            */
/* ------------------------------------------------------------------ */

/* x_{a,j} = -n h / 2 + j h */
static double lattice_x(int64_t n, double h, int64_t j) { return -0.5 * (double)n * h + (double)j * h; }

/* p_{a,k} = hbar 2 pi kappa_k / (n h), kappa_k = k if 2k < n else k - n
 * (for even n the Nyquist index n/2 maps to -n/2) */
static double lattice_p(int64_t n, double h, int64_t k, double hbar) {
    int64_t kap = (2 * k < n) ? k : k - n;
    return hbar * TWO_PI * (double)kap / ((double)n * h);
}

/* Multi-index (x fastest) of linear point index j. */
static void unravel(int64_t j, int ndim, const int64_t *dims, int64_t *idx) {
    for (int a = 0; a < ndim; ++a) {
        idx[a] = j % dims[a];
        j /= dims[a];
    }
}

static int64_t npoints(int ndim, const int64_t *dims) {
    int64_t N = 1;
    for (int a = 0; a < ndim; ++a) N *= dims[a];
    return N;
}

/* ------------------------------------------------------------------ */
/* Schroedinger split (Sec. 2.2)                                       */
/* ------------------------------------------------------------------ */

/* Real-space factor U_A1(t+tau, t, delta), Eq. 11 with Eq. 10a:
 *   psi_j <- exp(-i delta tau W_j / hbar) psi_j,  W_j = V_j - q x_j . E
 * (length gauge: the uniform field E enters the scalar potential as -x.E).
 * E = NULL means no field. */
static void schr_real_space(cplx *psi, const double *V, int ndim, const int64_t *dims,
                            const double *h, double charge, double hbar, double tau,
                            double delta, const double *E) {
    const int64_t N = npoints(ndim, dims);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t j = 0; j < N; ++j) {
        int64_t idx[3];
        unravel(j, ndim, dims, idx);
        double W = V ? V[j] : 0.0;
        if (E) {
            for (int a = 0; a < ndim; ++a) W -= charge * lattice_x(dims[a], h[a], idx[a]) * E[a];
        }
        double ang = -delta * tau * W / hbar;
        psi[j] *= cos(ang) + I * sin(ang);
    }
}

/* Momentum-space factor U~_A2(t+tau, t, 1), Eq. 13 with Eq. 10b.  A = NULL
 * (length gauge, or no field):
 *   psi~_k <- exp(-i tau |p_k|^2 / (2 m hbar)) psi~_k
 * Velocity gauge, A = the vector potential of this step (its midpoint value,
 * so that the time integral of Eq. 13 is tau times the integrand there):
 *   psi~_k <- exp(-i tau |p_k - q A|^2 / (2 m hbar)) psi~_k              */
static void schr_momentum_space(cplx *psit, int ndim, const int64_t *dims, const double *h,
                                double mass, double charge, double hbar, double tau, const double *A) {
    const int64_t N = npoints(ndim, dims);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t k = 0; k < N; ++k) {
        int64_t idx[3];
        unravel(k, ndim, dims, idx);
        double p2 = 0.0;
        for (int a = 0; a < ndim; ++a) {
            double p = lattice_p(dims[a], h[a], idx[a], hbar);
            if (A) p -= charge * A[a];
            p2 += p * p;
        }
        double ang = -tau * p2 / (2.0 * mass * hbar);
        psit[k] *= cos(ang) + I * sin(ang);
    }
}

/* n_steps Strang steps (Eq. 8).  field: n_steps x ndim samples (midpoint
 * of each step) or NULL; gauge 0: electric field E in the real-space factor
 * (length gauge, Eq. 11 with q phi = V - q x.E); gauge 1: vector potential A
 * in the momentum-space factor (velocity gauge, Eq. 13). */
int orc_schr_propagate_gauge(cplx *psi, const double *V, int ndim, const int64_t *dims,
                             const double *h, double mass, double charge, double hbar, double tau,
                             int64_t n_steps, const double *field, int gauge) {
    if (ndim < 1 || ndim > 3 || gauge < 0 || gauge > 1) return -1;
    for (int a = 0; a < ndim; ++a)
        if (!orc_size_ok(dims[a])) return -1;
    for (int64_t n = 0; n < n_steps; ++n) {
        const double *F = field ? field + n * ndim : NULL;
        const double *E = gauge == 0 ? F : NULL;
        const double *A = gauge == 1 ? F : NULL;
        schr_real_space(psi, V, ndim, dims, h, charge, hbar, tau, 0.5, E);
        orc_fftn(psi, ndim, dims, -1);
        schr_momentum_space(psi, ndim, dims, h, mass, charge, hbar, tau, A);
        orc_fftn(psi, ndim, dims, +1);
        schr_real_space(psi, V, ndim, dims, h, charge, hbar, tau, 0.5, E);
    }
    return 0;
}

int orc_schr_propagate(cplx *psi, const double *V, int ndim, const int64_t *dims,
                       const double *h, double mass, double charge, double hbar, double tau,
                       int64_t n_steps, const double *field) {
    return orc_schr_propagate_gauge(psi, V, ndim, dims, h, mass, charge, hbar, tau, n_steps, field, 0);
}

/* ------------------------------------------------------------------ */
/* Dirac split (Sec. 2.3), four components, d = 2 or 3                 */
/* ------------------------------------------------------------------ */

/* alpha_1, alpha_2, alpha_3 and beta in the Dirac representation, Eq. 16. */
static void dirac_matrices(cplx alpha[3][4][4], cplx beta[4][4]) {
    memset(alpha, 0, sizeof(cplx) * 48);
    memset(beta, 0, sizeof(cplx) * 16);
    /* alpha_1 */
    alpha[0][0][3] = 1; alpha[0][1][2] = 1; alpha[0][2][1] = 1; alpha[0][3][0] = 1;
    /* alpha_2 */
    alpha[1][0][3] = -I; alpha[1][1][2] = I; alpha[1][2][1] = -I; alpha[1][3][0] = I;
    /* alpha_3 */
    alpha[2][0][2] = 1; alpha[2][1][3] = -1; alpha[2][2][0] = 1; alpha[2][3][1] = -1;
    /* beta */
    beta[0][0] = 1; beta[1][1] = 1; beta[2][2] = -1; beta[3][3] = -1;
}

void orc_dirac_alpha_beta(double *out /* 4 x 16 complex: alpha1..3, beta */) {
    cplx al[3][4][4], be[4][4];
    dirac_matrices(al, be);
    cplx *o = (cplx *)out;
    memcpy(o, al, sizeof(cplx) * 48);
    memcpy(o + 48, be, sizeof(cplx) * 16);
}

static void mat4_mul(const cplx A[4][4], const cplx B[4][4], cplx C[4][4]) {
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += A[i][k] * B[k][j];
            C[i][j] = s;
        }
}

/* u(p) of Eq. 30 with d_+- of Eq. 29:
 *   d_+-(p) = ( 1/2 +- 1 / (2 sqrt(1 + p^2/(m c)^2)) )^{1/2}
 *   u(p)   = d_+ + d_- sum_i (p_i/|p|) beta alpha_i
 * At p = 0 the second term is absent (d_-(0) = 0). */
static void dirac_u(const double *p, int ndim, double mass, double c, cplx u[4][4]) {
    cplx al[3][4][4], be[4][4];
    dirac_matrices(al, be);
    double p2 = 0.0;
    for (int a = 0; a < ndim; ++a) p2 += p[a] * p[a];
    const double root = sqrt(1.0 + p2 / ((mass * c) * (mass * c)));
    const double dp = sqrt(0.5 + 0.5 / root);
    const double dm = sqrt(0.5 - 0.5 / root);
    const double pabs = sqrt(p2);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) u[i][j] = (i == j) ? dp : 0.0;
    if (pabs > 0.0) {
        for (int a = 0; a < ndim; ++a) {
            cplx ba[4][4];
            mat4_mul((const cplx(*)[4])be, (const cplx(*)[4])al[a], ba);
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) u[i][j] += dm * (p[a] / pabs) * ba[i][j];
        }
    }
}

void orc_dirac_u(const double *p, int ndim, double mass, double c, double *out /* 16 complex */) {
    cplx u[4][4];
    dirac_u(p, ndim, mass, c, u);
    memcpy(out, u, sizeof(cplx) * 16);
}

/* Free Dirac Hamiltonian in momentum space, c sum_i alpha_i p_i + m c^2 beta
 * (Eq. 28). */
static void dirac_h(const double *p, int ndim, double mass, double c, cplx H[4][4]) {
    cplx al[3][4][4], be[4][4];
    dirac_matrices(al, be);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = mass * c * c * be[i][j];
            for (int a = 0; a < ndim; ++a) s += c * p[a] * al[a][i][j];
            H[i][j] = s;
        }
}

void orc_dirac_h(const double *p, int ndim, double mass, double c, double *out) {
    cplx H[4][4];
    dirac_h(p, ndim, mass, c, H);
    memcpy(out, H, sizeof(cplx) * 16);
}

/* Kinetic factor of Eq. 33 applied to one spinor v (in place):
 *   v <- u^dagger diag(e^{-iE tau/hbar}, e^{-iE tau/hbar}, e^{iE tau/hbar}, e^{iE tau/hbar}) u v
 * with E(p) = sqrt(m^2 c^4 + p^2 c^2) (Eq. 32). */
static void dirac_kinetic_apply(const double *p, int ndim, double mass, double c, double hbar,
                                double tau, cplx v[4]) {
    cplx u[4][4];
    dirac_u(p, ndim, mass, c, u);
    double p2 = 0.0;
    for (int a = 0; a < ndim; ++a) p2 += p[a] * p[a];
    const double E = sqrt(mass * mass * c * c * c * c + p2 * c * c);
    const double ang = E * tau / hbar;
    const cplx em = cos(ang) - I * sin(ang), ep = cos(ang) + I * sin(ang);
    cplx w[4];
    for (int i = 0; i < 4; ++i) {
        cplx s = 0;
        for (int k = 0; k < 4; ++k) s += u[i][k] * v[k];
        w[i] = s;
    }
    w[0] *= em; w[1] *= em; w[2] *= ep; w[3] *= ep;
    for (int i = 0; i < 4; ++i) {
        cplx s = 0;
        for (int k = 0; k < 4; ++k) s += conj(u[k][i]) * w[k];
        v[i] = s;
    }
}

/* The 4x4 matrix of Eq. 33 (for the tests). */
void orc_dirac_kinetic_matrix(const double *p, int ndim, double mass, double c, double hbar,
                              double tau, double *out) {
    cplx M[4][4];
    for (int j = 0; j < 4; ++j) {
        cplx v[4] = {0, 0, 0, 0};
        v[j] = 1.0;
        dirac_kinetic_apply(p, ndim, mass, c, hbar, tau, v);
        for (int i = 0; i < 4; ++i) M[i][j] = v[i];
    }
    memcpy(out, M, sizeof(cplx) * 16);
}

/* Real-space mixing U_A1,2(t+tau, t, delta) of Eq. 26 for a uniform vector
 * potential, with Abar_i = int A_i dt' = A_i tau (Eq. 25a, midpoint rule) and
 * Abar = |Abar| (Eq. 25b).  It is exp(i delta q c sum_i alpha_i Abar_i / hbar)
 * (Eq. 20b in Eq. 5), which by Eq. 23 equals
 *   cos(theta) + i sum_i (Abar_i/Abar) alpha_i sin(theta),  theta = delta q c Abar / hbar;
 * for the electron, q = -1, this is the printed form of Eq. 26.
 * At Abar = 0 the matrix is the identity. */
static void dirac_mixing(const double *A, int ndim, double charge, double c, double hbar,
                         double tau, double delta, cplx R[4][4]) {
    cplx al[3][4][4], be[4][4];
    dirac_matrices(al, be);
    double Ab[3] = {0, 0, 0}, Aabs2 = 0.0;
    for (int a = 0; a < ndim; ++a) {
        Ab[a] = A ? A[a] * tau : 0.0;
        Aabs2 += Ab[a] * Ab[a];
    }
    const double Aabs = sqrt(Aabs2);
    const double theta = delta * charge * c * Aabs / hbar;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) R[i][j] = (i == j) ? cos(theta) : 0.0;
    if (Aabs > 0.0) {
        for (int a = 0; a < ndim; ++a)
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) R[i][j] += I * (Ab[a] / Aabs) * al[a][i][j] * sin(theta);
    }
}

void orc_dirac_mixing_matrix(const double *A, int ndim, double charge, double c, double hbar,
                             double tau, double delta, double *out) {
    cplx R[4][4];
    dirac_mixing(A, ndim, charge, c, hbar, tau, delta, R);
    memcpy(out, R, sizeof(cplx) * 16);
}

/* U_A1(t+tau, t, 1/2) = U_A1,1 U_A1,2 (Eqs. 21, 22, 26) on all points:
 *   psi_j <- exp(-i tau V_j / (2 hbar)) R psi_j                             */
static void dirac_real_space(cplx *psi, const double *V, int64_t N, const cplx R[4][4],
                             double hbar, double tau) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t j = 0; j < N; ++j) {
        cplx v[4], w[4];
        for (int c = 0; c < 4; ++c) v[c] = psi[c * N + j];
        for (int i = 0; i < 4; ++i) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += R[i][k] * v[k];
            w[i] = s;
        }
        double ang = -0.5 * tau * (V ? V[j] : 0.0) / hbar;
        cplx ph = cos(ang) + I * sin(ang);
        for (int c = 0; c < 4; ++c) psi[c * N + j] = ph * w[c];
    }
}

static void dirac_momentum_space(cplx *psit, int ndim, const int64_t *dims, const double *h,
                                 double mass, double c, double hbar, double tau) {
    const int64_t N = npoints(ndim, dims);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t k = 0; k < N; ++k) {
        int64_t idx[3];
        double p[3] = {0, 0, 0};
        unravel(k, ndim, dims, idx);
        for (int a = 0; a < ndim; ++a) p[a] = lattice_p(dims[a], h[a], idx[a], hbar);
        cplx v[4];
        for (int cc = 0; cc < 4; ++cc) v[cc] = psit[cc * N + k];
        dirac_kinetic_apply(p, ndim, mass, c, hbar, tau, v);
        for (int cc = 0; cc < 4; ++cc) psit[cc * N + k] = v[cc];
    }
}

/* n_steps Strang steps (Eq. 8) of the four-component Dirac equation, d = 2
 * or 3.  field: n_steps x ndim vector-potential samples (midpoints) or NULL. */
int orc_dirac_propagate(cplx *psi, const double *V, int ndim, const int64_t *dims,
                        const double *h, double mass, double charge, double hbar, double c,
                        double tau, int64_t n_steps, const double *field) {
    if (ndim < 2 || ndim > 3) return -1;
    for (int a = 0; a < ndim; ++a)
        if (!orc_size_ok(dims[a])) return -1;
    const int64_t N = npoints(ndim, dims);
    for (int64_t n = 0; n < n_steps; ++n) {
        cplx R[4][4];
        dirac_mixing(field ? field + n * ndim : NULL, ndim, charge, c, hbar, tau, 0.5, R);
        dirac_real_space(psi, V, N, (const cplx(*)[4])R, hbar, tau);
        for (int cc = 0; cc < 4; ++cc) orc_fftn(psi + cc * N, ndim, dims, -1);
        dirac_momentum_space(psi, ndim, dims, h, mass, c, hbar, tau);
        for (int cc = 0; cc < 4; ++cc) orc_fftn(psi + cc * N, ndim, dims, +1);
        dirac_real_space(psi, V, N, (const cplx(*)[4])R, hbar, tau);
    }
    return 0;
}

/* A vector potential that varies along x_1 (a plane-wave laser pulse
 * travelling along x_1, the scattering example of the paper's results): the
 * mixing of Eq. 26 then differs per lattice column, with Abar(x) = A(x_1, t)
 * tau.  field: n_steps x dims[0] x ndim samples, A at the step midpoint and
 * lattice column i of axis 0. */
int orc_dirac_propagate_profile(cplx *psi, const double *V, int ndim, const int64_t *dims,
                                const double *h, double mass, double charge, double hbar, double c,
                                double tau, int64_t n_steps, const double *field) {
    if (ndim < 2 || ndim > 3 || !field) return -1;
    for (int a = 0; a < ndim; ++a)
        if (!orc_size_ok(dims[a])) return -1;
    const int64_t N = npoints(ndim, dims), nx = dims[0];
    cplx(*R)[4][4] = (cplx(*)[4][4])malloc(sizeof(cplx) * 16 * (size_t)nx);
    for (int64_t n = 0; n < n_steps; ++n) {
        for (int64_t i = 0; i < nx; ++i)
            dirac_mixing(field + (n * nx + i) * ndim, ndim, charge, c, hbar, tau, 0.5, R[i]);
        for (int half = 0; half < 2; ++half) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
            for (int64_t j = 0; j < N; ++j) {
                const cplx(*Rj)[4] = (const cplx(*)[4])R[j % nx];
                cplx v[4], w[4];
                for (int cc = 0; cc < 4; ++cc) v[cc] = psi[cc * N + j];
                for (int r = 0; r < 4; ++r) {
                    cplx s = 0;
                    for (int k = 0; k < 4; ++k) s += Rj[r][k] * v[k];
                    w[r] = s;
                }
                double ang = -0.5 * tau * (V ? V[j] : 0.0) / hbar;
                cplx ph = cos(ang) + I * sin(ang);
                for (int cc = 0; cc < 4; ++cc) psi[cc * N + j] = ph * w[cc];
            }
            if (half == 1) break;
            for (int cc = 0; cc < 4; ++cc) orc_fftn(psi + cc * N, ndim, dims, -1);
            dirac_momentum_space(psi, ndim, dims, h, mass, c, hbar, tau);
            for (int cc = 0; cc < 4; ++cc) orc_fftn(psi + cc * N, ndim, dims, +1);
        }
    }
    free(R);
    return 0;
}

/* ------------------------------------------------------------------ */
/* One-dimensional Dirac equation, two components (end of Sec. 2.3)    */
/* ------------------------------------------------------------------ */

/* The paper writes the 1D operators with alpha_1 and beta without printing
 * their 2x2 form; this oracle takes alpha_1 = sigma_x, beta = sigma_z (they
 * anticommute and square to one, as Eq. 15 requires). */
static void dirac1d_matrices(cplx al[2][2], cplx be[2][2]) {
    al[0][0] = 0; al[0][1] = 1; al[1][0] = 1; al[1][1] = 0;
    be[0][0] = 1; be[0][1] = 0; be[1][0] = 0; be[1][1] = -1;
}

/* u(p) = d_+ + d_- (p/|p|) beta alpha_1 with d_+- of Eq. 29: the 2x2 form of
 * Eq. 30, which turns c alpha_1 p + m c^2 beta into diag(E, -E). */
static void dirac1d_u(double p, double mass, double c, cplx u[2][2]) {
    cplx al[2][2], be[2][2];
    dirac1d_matrices(al, be);
    const double root = sqrt(1.0 + p * p / ((mass * c) * (mass * c)));
    const double dp = sqrt(0.5 + 0.5 / root);
    const double dm = sqrt(0.5 - 0.5 / root);
    const double sgn = p > 0.0 ? 1.0 : (p < 0.0 ? -1.0 : 0.0);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            cplx ba = 0;
            for (int k = 0; k < 2; ++k) ba += be[i][k] * al[k][j];
            u[i][j] = (i == j ? dp : 0.0) + dm * sgn * ba;
        }
}

void orc_dirac1d_u(double p, double mass, double c, double *out /* 4 complex */) {
    cplx u[2][2];
    dirac1d_u(p, mass, c, u);
    memcpy(out, u, sizeof(cplx) * 4);
}

/* H = c alpha_1 p + m c^2 beta (Eq. 28 in one dimension). */
static void dirac1d_h(double p, double mass, double c, cplx H[2][2]) {
    cplx al[2][2], be[2][2];
    dirac1d_matrices(al, be);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) H[i][j] = c * p * al[i][j] + mass * c * c * be[i][j];
}

void orc_dirac1d_h(double p, double mass, double c, double *out) {
    cplx H[2][2];
    dirac1d_h(p, mass, c, H);
    memcpy(out, H, sizeof(cplx) * 4);
}

/* Momentum-space factor of the 1D Dirac equation:
 *   v <- u^dagger diag(e^{-iE tau/hbar}, e^{iE tau/hbar}) u v,  E = sqrt(m^2 c^4 + p^2 c^2). */
static void dirac1d_kinetic_apply(double p, double mass, double c, double hbar, double tau, cplx v[2]) {
    cplx u[2][2];
    dirac1d_u(p, mass, c, u);
    const double E = sqrt(mass * mass * c * c * c * c + p * p * c * c);
    const double ang = E * tau / hbar;
    cplx w[2];
    for (int i = 0; i < 2; ++i) w[i] = u[i][0] * v[0] + u[i][1] * v[1];
    w[0] *= cos(ang) - I * sin(ang);
    w[1] *= cos(ang) + I * sin(ang);
    for (int i = 0; i < 2; ++i) v[i] = conj(u[0][i]) * w[0] + conj(u[1][i]) * w[1];
}

/* Real-space half factor: exp(-i tau V/(2 hbar)) times the 1D mixing
 * R = cos(theta) + i alpha_1 sin(theta), theta = delta q c Abar / hbar,
 * Abar = A tau (midpoint rule); for q = -1 this is the printed form. */
static void dirac1d_real_space(cplx *psi, const double *V, int64_t n, const double *A, double charge,
                               double c, double hbar, double tau) {
    cplx al[2][2], be[2][2];
    dirac1d_matrices(al, be);
    const double theta = 0.5 * charge * c * (A ? *A * tau : 0.0) / hbar;
    cplx R[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) R[i][j] = (i == j ? cos(theta) : 0.0) + I * sin(theta) * al[i][j];
    for (int64_t j = 0; j < n; ++j) {
        const cplx a = psi[j], b = psi[n + j];
        const double ang = -0.5 * tau * (V ? V[j] : 0.0) / hbar;
        const cplx ph = cos(ang) + I * sin(ang);
        psi[j] = ph * (R[0][0] * a + R[0][1] * b);
        psi[n + j] = ph * (R[1][0] * a + R[1][1] * b);
    }
}

/* n_steps Strang steps (Eq. 8) of the two-component 1D Dirac equation:
 * psi is [2][n]; field: n_steps vector-potential samples A_1 (midpoints) or NULL. */
int orc_dirac1d_propagate(cplx *psi, const double *V, int64_t n, double h, double mass, double charge,
                          double hbar, double c, double tau, int64_t n_steps, const double *field) {
    if (!orc_size_ok(n)) return -1;
    const int64_t dims[1] = {n};
    for (int64_t s = 0; s < n_steps; ++s) {
        const double *A = field ? field + s : NULL;
        dirac1d_real_space(psi, V, n, A, charge, c, hbar, tau);
        orc_fftn(psi, 1, dims, -1);
        orc_fftn(psi + n, 1, dims, -1);
        for (int64_t k = 0; k < n; ++k) {
            cplx v[2] = {psi[k], psi[n + k]};
            dirac1d_kinetic_apply(lattice_p(n, h, k, hbar), mass, c, hbar, tau, v);
            psi[k] = v[0];
            psi[n + k] = v[1];
        }
        orc_fftn(psi, 1, dims, +1);
        orc_fftn(psi + n, 1, dims, +1);
        dirac1d_real_space(psi, V, n, A, charge, c, hbar, tau);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Reductions                                                          */
/* ------------------------------------------------------------------ */

typedef struct {
    double s, c;
} kahan;

static void kahan_add(kahan *k, double x) {
    double y = x - k->c;
    double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

static double cell_volume(int ndim, const double *h) {
    double dv = 1.0;
    for (int a = 0; a < ndim; ++a) dv *= h[a];
    return dv;
}

/* norm = dV sum_{c,j} |psi_{c,j}|^2 */
double orc_norm(const cplx *psi, int ndim, const int64_t *dims, const double *h, int comps) {
    const int64_t N = npoints(ndim, dims) * comps;
    kahan k = {0, 0};
    for (int64_t j = 0; j < N; ++j) kahan_add(&k, creal(psi[j]) * creal(psi[j]) + cimag(psi[j]) * cimag(psi[j]));
    return k.s * cell_volume(ndim, h);
}

/* Field-free energy <H0> = <T> + <V>:
 *   <V> = dV sum_j V_j sum_c |psi_{c,j}|^2
 *   <T> = (dV / N) sum_k psi~_k^dagger T(p_k) psi~_k
 * with T = |p|^2/(2m) (Schroedinger) or T = c alpha.p + m c^2 beta (Dirac,
 * Eq. 28).  dV/N turns the unnormalised DFT sum into the same measure
 * (Parseval). */
double orc_energy(const cplx *psi, const double *V, int ndim, const int64_t *dims,
                  const double *h, int comps, double mass, double hbar, double c) {
    const int64_t N = npoints(ndim, dims);
    const double dV = cell_volume(ndim, h);
    kahan kv = {0, 0}, kt = {0, 0};
    if (V) {
        for (int64_t j = 0; j < N; ++j) {
            double r = 0.0;
            for (int cc = 0; cc < comps; ++cc) {
                cplx z = psi[cc * N + j];
                r += creal(z) * creal(z) + cimag(z) * cimag(z);
            }
            kahan_add(&kv, V[j] * r);
        }
    }
    cplx *pt = (cplx *)malloc(sizeof(cplx) * (size_t)(N * comps));
    memcpy(pt, psi, sizeof(cplx) * (size_t)(N * comps));
    for (int cc = 0; cc < comps; ++cc) orc_fftn(pt + cc * N, ndim, dims, -1);
    for (int64_t k = 0; k < N; ++k) {
        int64_t idx[3];
        double p[3] = {0, 0, 0}, p2 = 0.0;
        unravel(k, ndim, dims, idx);
        for (int a = 0; a < ndim; ++a) {
            p[a] = lattice_p(dims[a], h[a], idx[a], hbar);
            p2 += p[a] * p[a];
        }
        if (comps == 1) {
            cplx z = pt[k];
            kahan_add(&kt, (p2 / (2.0 * mass)) * (creal(z) * creal(z) + cimag(z) * cimag(z)));
        } else if (comps == 2) {
            cplx H[2][2];
            dirac1d_h(p[0], mass, c, H);
            cplx s = 0;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) s += conj(pt[i * N + k]) * H[i][j] * pt[j * N + k];
            kahan_add(&kt, creal(s));
        } else {
            cplx H[4][4];
            dirac_h(p, ndim, mass, c, H);
            cplx s = 0;
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) s += conj(pt[i * N + k]) * H[i][j] * pt[j * N + k];
            kahan_add(&kt, creal(s));
        }
    }
    free(pt);
    return dV * kv.s + (dV / (double)N) * kt.s;
}
