/*
 * Plain FP64 CPU oracle for the even-odd preconditioned Wilson matrix.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference legs may load this library. The CUDA
 * product path never calls it and shares no code, header or table with it.
 *
 * What it computes (Kanamori, Nitadori, Matsufuru, "Wilson matrix kernel for
 * lattice QCD on A64FX architecture", arXiv:2303.08609):
 *
 *   D_W(x,y) = delta_{x,y} - kappa * sum_mu [ (1 - gamma_mu) U_mu(x) delta_{x+mu,y}
 *                                         + (1 + gamma_mu) U_mu^dag(x-mu) delta_{x-mu,y} ]
 *                                                               (Sec. 2, Eq. 1 and its footnote)
 *   H = the bracketed hopping sum without -kappa, so D_eo = -kappa H_eo and
 *       D_oe = -kappa H_oe, and since D_ee = D_oo = 1 (Sec. 2, after Eq. 5)
 *   M_eo = 1 - D_eo D_oe = 1 - kappa^2 H_eo H_oe           (Sec. 2, Eq. 4)
 *
 * Everything is written out in the plainest form: full 4x4 gamma matrices and
 * full 3x3 link multiplications on all four spin components (no half-spinor
 * projection shortcut), loops over lexicographic sites with the parity test
 * "x+y+z+t even" (Sec. 3.3, Fig. 4), periodic boundaries in all directions.
 *
 * Readings of points the paper leaves open (each is listed in the design notes):
 *  - gamma basis: Euclidean chiral basis, gamma_k = [[0,-i s_k],[i s_k,0]]
 *    (k = x,y,z; s_k the Pauli matrices), gamma_t = [[0,1],[1,0]],
 *    gamma_5 = gamma_x gamma_y gamma_z gamma_t = diag(1,1,-1,-1);
 *  - projector signs follow Eq. 1 / its footnote: (1 - gamma) with the forward
 *    neighbour, (1 + gamma) with the backward one. Fig. 2 pairs them the other
 *    way round; the two differ by conjugation with gamma_5 (tested);
 *  - U_mu^dag(x - mu) is the conjugate transpose of the link stored at x - mu
 *    (footnote of Eq. 1: (U_mu)^*_{ba}(x - mu));
 *  - single-parity arrays are compacted in x (Sec. 3.3): the site with
 *    lexicographic index ((t*Lz+z)*Ly+y)*Lx+x has parity index lex/2.
 *
 * Layouts (complex interleaved): gauge U[mu][lex][a][b]; spinor psi[i][spin][colour].
 *
 * Pins (tests marked "not gpu"): dense brute-force D_W at 4^4, adjoint identity,
 * gamma_5-hermiticity, free-field plane-wave closed form, gauge covariance,
 * sign-convention identity, Schur solve against the dense matrix, central
 * finite differences for the link gradient and the force.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ---------------------------------------------------------------- basis -- */

/* gamma[mu][row][col], mu = 0..3 for x, y, z, t (chiral basis, see header). */
static const cplx GAMMA[4][4][4] = {
    /* gamma_x: [[0, -i s1], [i s1, 0]] */
    {{0, 0, 0, -I}, {0, 0, -I, 0}, {0, I, 0, 0}, {I, 0, 0, 0}},
    /* gamma_y: [[0, -i s2], [i s2, 0]], -i s2 = [[0,-1],[1,0]] */
    {{0, 0, 0, -1}, {0, 0, 1, 0}, {0, 1, 0, 0}, {-1, 0, 0, 0}},
    /* gamma_z: [[0, -i s3], [i s3, 0]], -i s3 = diag(-i, i) */
    {{0, 0, -I, 0}, {0, 0, 0, I}, {I, 0, 0, 0}, {0, -I, 0, 0}},
    /* gamma_t: [[0, 1], [1, 0]] */
    {{0, 0, 1, 0}, {0, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}},
};

/* Exposes the basis so the tests can check its algebra. out: 16 complex. */
void oracle_gamma(int mu, double *out)
{
    cplx *o = (cplx *)out;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) o[4 * i + j] = GAMMA[mu][i][j];
}

/* P = 1 + s * gamma_mu (s = +1 or -1). */
static void projector(int mu, int s, cplx P[4][4])
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) P[i][j] = (i == j ? 1.0 : 0.0) + s * GAMMA[mu][i][j];
}

/* ------------------------------------------------------------- geometry -- */

static long vol(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords(const int L[4], long lex, int c[4])
{
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = (int)(lex % L[mu]);
        lex /= L[mu];
    }
}

static long lex_of(const int L[4], const int c[4])
{
    return ((long)(c[3] * L[2] + c[2]) * L[1] + c[1]) * L[0] + c[0];
}

/* lexicographic index of the site c + dir * mu-hat, periodic */
static long neighbour(const int L[4], const int c[4], int mu, int dir)
{
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] = (d[mu] + dir + L[mu]) % L[mu];
    return lex_of(L, d);
}

static int parity_of(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

/* ------------------------------------------------------ block algebra -- */

/* A hopping block is the 12x12 matrix P (x) W on spin (x) colour, where P is a
 * 4x4 spin matrix and W = U or U^dag for one 3x3 link U. apply_block computes
 * out += B v, or out += B^dag v when adjoint != 0, with B^dag = P^dag (x) W^dag
 * written out elementwise. */
static void apply_block(const cplx P[4][4], const cplx *U, int link_dag, int adjoint,
                        const cplx *v, cplx *out)
{
    cplx Ps[4][4], W[3][3];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) Ps[i][j] = adjoint ? conj(P[j][i]) : P[i][j];
    /* W = U (link_dag = 0) or U^dag (link_dag = 1); the block adjoint adds one more ^dag */
    int wdag = link_dag ^ adjoint;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) W[a][b] = wdag ? conj(U[3 * b + a]) : U[3 * a + b];
    for (int i = 0; i < 4; ++i)
        for (int a = 0; a < 3; ++a) {
            cplx s = 0;
            for (int j = 0; j < 4; ++j)
                for (int b = 0; b < 3; ++b) s += Ps[i][j] * W[a][b] * v[3 * j + b];
            out[3 * i + a] += s;
        }
}

/* ------------------------------------------------------------- hopping -- */

/* (H psi)(x) at one site x (lexicographic), psi on the opposite parity.
 * sign = +1 is Eq. 1; sign = -1 swaps the projectors (the Fig. 2 pairing). */
static void hop_site(const int L[4], const cplx *U, int sign, long x, const cplx *in, cplx *acc)
{
    const long V = vol(L);
    int c[4];
    coords(L, x, c);
    for (int k = 0; k < 12; ++k) acc[k] = 0;
    for (int mu = 0; mu < 4; ++mu) {
        cplx Pf[4][4], Pb[4][4];
        projector(mu, -sign, Pf); /* 1 - gamma_mu for sign = +1 */
        projector(mu, +sign, Pb); /* 1 + gamma_mu for sign = +1 */
        long yf = neighbour(L, c, mu, +1);
        long yb = neighbour(L, c, mu, -1);
        /* forward: (1 - gamma_mu) U_mu(x) psi(x + mu) */
        apply_block(Pf, U + 9 * (mu * V + x), 0, 0, in + 12 * (yf / 2), acc);
        /* backward: (1 + gamma_mu) U_mu^dag(x - mu) psi(x - mu) */
        apply_block(Pb, U + 9 * (mu * V + yb), 1, 0, in + 12 * (yb / 2), acc);
    }
}

/* (H^dag psi)(y) at one site y, written as the sum over x of H(x,y)^dag psi(x):
 * H(x,y) is non-zero for x = y - mu (forward block of x, link U_mu(y - mu)) and
 * for x = y + mu (backward block of x, link U_mu(y)^dag). */
static void hop_adj_site(const int L[4], const cplx *U, int sign, long y, const cplx *in,
                         cplx *acc)
{
    const long V = vol(L);
    int c[4];
    coords(L, y, c);
    for (int k = 0; k < 12; ++k) acc[k] = 0;
    for (int mu = 0; mu < 4; ++mu) {
        cplx Pf[4][4], Pb[4][4];
        projector(mu, -sign, Pf);
        projector(mu, +sign, Pb);
        long xm = neighbour(L, c, mu, -1); /* x = y - mu: forward block of x */
        long xp = neighbour(L, c, mu, +1); /* x = y + mu: backward block of x */
        apply_block(Pf, U + 9 * (mu * V + xm), 0, 1, in + 12 * (xm / 2), acc);
        apply_block(Pb, U + 9 * (mu * V + y), 1, 1, in + 12 * (xp / 2), acc);
    }
}

/* out[i] = (H psi) on all sites of parity out_parity; in on the other parity. */
void oracle_hop(const int *L, const double *Ud, int sign, int out_parity, double *outd,
                const double *ind)
{
    const cplx *U = (const cplx *)Ud, *in = (const cplx *)ind;
    cplx *out = (cplx *)outd;
    const long V = vol(L);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        int c[4];
        coords(L, x, c);
        if (parity_of(c) != out_parity) continue;
        hop_site(L, U, sign, x, in, out + 12 * (x / 2));
    }
}

/* out = (H^dag psi) on all sites of parity out_parity (explicit adjoint blocks). */
void oracle_hop_adj(const int *L, const double *Ud, int sign, int out_parity, double *outd,
                    const double *ind)
{
    const cplx *U = (const cplx *)Ud, *in = (const cplx *)ind;
    cplx *out = (cplx *)outd;
    const long V = vol(L);
#pragma omp parallel for schedule(static)
    for (long y = 0; y < V; ++y) {
        int c[4];
        coords(L, y, c);
        if (parity_of(c) != out_parity) continue;
        hop_adj_site(L, U, sign, y, in, out + 12 * (y / 2));
    }
}

/* ------------------------------------------------------------ M_eo ------- */

/* out_e = in_e - kappa^2 H_eo H_oe in_e (Eq. 4 with D_ee = D_oo = 1). */
void oracle_meo(const int *L, const double *U, double kappa, double *out_e, const double *in_e)
{
    const long Vh = vol(L) / 2;
    double *tmp = (double *)malloc(sizeof(double) * 24 * Vh);
    oracle_hop(L, U, +1, 1, tmp, in_e);   /* H_oe: even -> odd */
    oracle_hop(L, U, +1, 0, out_e, tmp);  /* H_eo: odd -> even */
    for (long k = 0; k < 24 * Vh; ++k) out_e[k] = in_e[k] - kappa * kappa * out_e[k];
    free(tmp);
}

/* out_e = M_eo^dag in_e = in_e - kappa^2 (H_eo H_oe)^dag in_e
 *       = in_e - kappa^2 H_oe^dag H_eo^dag in_e, with explicit adjoint blocks. */
void oracle_meo_dag(const int *L, const double *U, double kappa, double *out_e,
                    const double *in_e)
{
    const long Vh = vol(L) / 2;
    double *tmp = (double *)malloc(sizeof(double) * 24 * Vh);
    oracle_hop_adj(L, U, +1, 1, tmp, in_e);   /* H_eo^dag: even -> odd */
    oracle_hop_adj(L, U, +1, 0, out_e, tmp);  /* H_oe^dag: odd -> even */
    for (long k = 0; k < 24 * Vh; ++k) out_e[k] = in_e[k] - kappa * kappa * out_e[k];
    free(tmp);
}

/* M_eo with the projector signs swapped (sign = -1): used to test the
 * sign-convention identity M[-gamma] = gamma_5 M[gamma] gamma_5. */
void oracle_meo_sign(const int *L, const double *U, double kappa, int sign, double *out_e,
                     const double *in_e)
{
    const long Vh = vol(L) / 2;
    double *tmp = (double *)malloc(sizeof(double) * 24 * Vh);
    oracle_hop(L, U, sign, 1, tmp, in_e);
    oracle_hop(L, U, sign, 0, out_e, tmp);
    for (long k = 0; k < 24 * Vh; ++k) out_e[k] = in_e[k] - kappa * kappa * out_e[k];
    free(tmp);
}

/* even lexicographic site with parity index i */
static long even_lex(const int L[4], long i)
{
    int c[4];
    coords(L, 2 * i, c);
    return parity_of(c) == 0 ? 2 * i : 2 * i + 1;
}

/* M_eo (dag = 0) or M_eo^dag (dag = 1) at selected even sites only: for each
 * listed parity index, the odd intermediate is computed at the 8 neighbours
 * that the outer hop reads, then the outer hop (the same blocks as hop_site /
 * hop_adj_site, applied to those 8 values) and the diagonal term.
 * out: nsites x 12 complex. Used to check very large lattices site by site. */
void oracle_meo_sites(const int *L, const double *Ud, double kappa, int dag, const double *ind,
                      long nsites, const long *sites, double *outd)
{
    const cplx *U = (const cplx *)Ud, *in = (const cplx *)ind;
    cplx *out = (cplx *)outd;
    const long V = vol(L);
#pragma omp parallel for schedule(dynamic, 4)
    for (long n = 0; n < nsites; ++n) {
        long x = even_lex(L, sites[n]);
        int c[4];
        coords(L, x, c);
        cplx tf[4][12], tb[4][12], acc[12];
        for (int mu = 0; mu < 4; ++mu) {
            long yf = neighbour(L, c, mu, +1), yb = neighbour(L, c, mu, -1);
            if (dag) {
                hop_adj_site(L, U, +1, yf, in, tf[mu]);
                hop_adj_site(L, U, +1, yb, in, tb[mu]);
            } else {
                hop_site(L, U, +1, yf, in, tf[mu]);
                hop_site(L, U, +1, yb, in, tb[mu]);
            }
        }
        for (int k = 0; k < 12; ++k) acc[k] = 0;
        for (int mu = 0; mu < 4; ++mu) {
            cplx Pf[4][4], Pb[4][4];
            projector(mu, -1, Pf);
            projector(mu, +1, Pb);
            long yb = neighbour(L, c, mu, -1);
            if (dag) {
                apply_block(Pf, U + 9 * (mu * V + yb), 0, 1, tb[mu], acc);
                apply_block(Pb, U + 9 * (mu * V + x), 1, 1, tf[mu], acc);
            } else {
                apply_block(Pf, U + 9 * (mu * V + x), 0, 0, tf[mu], acc);
                apply_block(Pb, U + 9 * (mu * V + yb), 1, 0, tb[mu], acc);
            }
        }
        for (int k = 0; k < 12; ++k)
            out[12 * n + k] = in[12 * (x / 2) + k] - kappa * kappa * acc[k];
    }
}

/* ----------------------------------------------------- link gradient -- */

/* Spin-traced colour outer product: G[a][b] += f * sum_j p[j][a] conj(q[j][b]). */
static void outer_acc(cplx *G, cplx f, const cplx *p, const cplx *q)
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            cplx s = 0;
            for (int j = 0; j < 4; ++j) s += p[3 * j + a] * conj(q[3 * j + b]);
            G[3 * a + b] += f * s;
        }
}

/* w = P v for a 4x4 spin matrix P */
static void spin_apply(const cplx P[4][4], const cplx *v, cplx *w)
{
    for (int i = 0; i < 4; ++i)
        for (int a = 0; a < 3; ++a) {
            cplx s = 0;
            for (int j = 0; j < 4; ++j) s += P[i][j] * v[3 * j + a];
            w[3 * i + a] = s;
        }
}

/* Gradient of L = Re<g, M_eo phi> with respect to every link, as the complex
 * matrix G_mu(x) with dL = Re sum conj(G_mu(x)_ab) dU_mu(x)_ab (the convention
 * of a real loss of complex inputs: G = dL/dRe U + i dL/dIm U).
 *
 * With t = H_oe phi and w = H_eo^dag g:
 *   dL = -kappa^2 ( Re<g, dH_eo t> + Re<w, dH_oe phi> ).
 * Differentiating the two terms of Eq. 1 at a link U_mu(x):
 *   forward term of site x, (1 - gamma) U b(x+mu), seen from output vector a:
 *       G += sum_spin [(1 - gamma) a(x)] (x) conj(b(x + mu))
 *   backward term of site x+mu, (1 + gamma) U^dag b(x):
 *       G += sum_spin b(x) (x) conj([(1 + gamma) a(x + mu)])
 * For x even the link is the forward link of H_eo (a = g, b = t) and the
 * backward link of H_oe (a = w, b = phi); for x odd the other way round.
 * G: [mu][lex][3][3] complex. */
void oracle_link_grad(const int *L, const double *Ud, double kappa, const double *gd,
                      const double *phid, double *Gd)
{
    const cplx *g = (const cplx *)gd, *phi = (const cplx *)phid;
    cplx *G = (cplx *)Gd;
    const long V = vol(L);
    const long Vh = V / 2;
    double *t = (double *)malloc(sizeof(double) * 24 * Vh);
    double *w = (double *)malloc(sizeof(double) * 24 * Vh);
    oracle_hop(L, Ud, +1, 1, t, phid);    /* t = H_oe phi (odd) */
    oracle_hop_adj(L, Ud, +1, 1, w, gd);  /* w = H_eo^dag g (odd) */
    const cplx *tc = (const cplx *)t, *wc = (const cplx *)w;
    const cplx f = -kappa * kappa;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        int c[4];
        coords(L, x, c);
        const int px = parity_of(c);
        for (int mu = 0; mu < 4; ++mu) {
            cplx *Gl = G + 9 * (mu * V + x);
            for (int k = 0; k < 9; ++k) Gl[k] = 0;
            cplx Pm[4][4], Pp[4][4], tmp[12];
            projector(mu, -1, Pm); /* 1 - gamma_mu */
            projector(mu, +1, Pp); /* 1 + gamma_mu */
            long xf = neighbour(L, c, mu, +1);
            if (px == 0) {
                /* H_eo forward at even x: a = g(x), b = t(x+mu) */
                spin_apply(Pm, g + 12 * (x / 2), tmp);
                outer_acc(Gl, f, tmp, tc + 12 * (xf / 2));
                /* H_oe backward at odd x+mu: b = phi(x), a = w(x+mu) */
                spin_apply(Pp, wc + 12 * (xf / 2), tmp);
                outer_acc(Gl, f, phi + 12 * (x / 2), tmp);
            } else {
                /* H_eo backward at even x+mu: b = t(x), a = g(x+mu) */
                spin_apply(Pp, g + 12 * (xf / 2), tmp);
                outer_acc(Gl, f, tc + 12 * (x / 2), tmp);
                /* H_oe forward at odd x: a = w(x), b = phi(x+mu) */
                spin_apply(Pm, wc + 12 * (x / 2), tmp);
                outer_acc(Gl, f, tmp, phi + 12 * (xf / 2));
            }
        }
    }
    free(t);
    free(w);
}

/* Pseudofermion force of S = |M_eo phi|^2: the traceless anti-Hermitian F_mu(x)
 * with dS/d(eps) = Re tr(X^dag F) for every traceless anti-Hermitian X under
 * U_mu(x) -> exp(eps X) U_mu(x). With G the link gradient of S (g = 2 M_eo phi),
 * dS = Re tr(X U G^dag) eps, hence F = TA(G U^dag) with
 * TA(W) = (W - W^dag)/2 - tr(W - W^dag)/6. Also returns dS/dphi = 2 M^dag M phi
 * when dphi is not NULL. F: [mu][lex][3][3] complex. */
void oracle_force(const int *L, const double *Ud, double kappa, const double *phid,
                  double *Fd, double *dphid)
{
    const cplx *U = (const cplx *)Ud;
    cplx *F = (cplx *)Fd;
    const long V = vol(L);
    const long Vh = V / 2;
    double *chi = (double *)malloc(sizeof(double) * 24 * Vh);
    double *G = (double *)malloc(sizeof(double) * 18 * 4 * V);
    oracle_meo(L, Ud, kappa, chi, phid);
    for (long k = 0; k < 24 * Vh; ++k) chi[k] *= 2.0; /* dS/dchi = 2 chi */
    oracle_link_grad(L, Ud, kappa, chi, phid, G);
    const cplx *Gc = (const cplx *)G;
    for (long l = 0; l < 4 * V; ++l) {
        const cplx *Ul = U + 9 * l, *Gl = Gc + 9 * l;
        cplx W[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                cplx s = 0;
                for (int k = 0; k < 3; ++k) s += Gl[3 * a + k] * conj(Ul[3 * b + k]);
                W[3 * a + b] = s;
            }
        cplx tr = 0;
        for (int a = 0; a < 3; ++a) tr += W[4 * a] - conj(W[4 * a]);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                F[9 * l + 3 * a + b] =
                    0.5 * (W[3 * a + b] - conj(W[3 * b + a])) - (a == b ? tr / 6.0 : 0.0);
    }
    if (dphid) oracle_meo_dag(L, Ud, kappa, dphid, chi); /* 2 M^dag chi */
    free(chi);
    free(G);
}

/* ------------------------------------------------------------- solver -- */

static cplx dot(long n, const cplx *a, const cplx *b)
{
    cplx s = 0;
    for (long k = 0; k < n; ++k) s += conj(a[k]) * b[k];
    return s;
}

/* A v = M_eo^dag M_eo v */
static void normal_op(const int *L, const double *U, double kappa, double *out, const double *v,
                      double *tmp)
{
    oracle_meo(L, U, kappa, tmp, v);
    oracle_meo_dag(L, U, kappa, out, tmp);
}

/* Conjugate gradient on A = M_eo^dag M_eo (Hermitian positive definite), FP64,
 * x in: initial guess, out: solution. Stops when |r|/|b| <= tol on the iterated
 * residual or after maxiter iterations; relres_out receives the true relative
 * residual |b - A x| / |b| recomputed from scratch. Returns 0 when the true
 * residual meets tol, 1 otherwise, -1 when out of memory. */
int oracle_cg(const int *L, const double *U, double kappa, const double *bd, double *xd,
              double tol, int maxiter, int *iters_out, double *relres_out)
{
    const long n = 12 * (vol(L) / 2);
    cplx *b = (cplx *)bd, *x = (cplx *)xd;
    cplx *r = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n);
    cplx *Ap = malloc(sizeof(cplx) * n), *tmp = malloc(sizeof(cplx) * n);
    if (!r || !p || !Ap || !tmp) {
        free(r);
        free(p);
        free(Ap);
        free(tmp);
        return -1;
    }
    normal_op(L, U, kappa, (double *)Ap, xd, (double *)tmp);
    for (long k = 0; k < n; ++k) r[k] = b[k] - Ap[k];
    for (long k = 0; k < n; ++k) p[k] = r[k];
    double bb = creal(dot(n, b, b));
    double rr = creal(dot(n, r, r));
    int it = 0;
    while (it < maxiter && sqrt(rr / bb) > tol) {
        normal_op(L, U, kappa, (double *)Ap, (double *)p, (double *)tmp);
        double pAp = creal(dot(n, p, Ap));
        double alpha = rr / pAp;
        for (long k = 0; k < n; ++k) {
            x[k] += alpha * p[k];
            r[k] -= alpha * Ap[k];
        }
        double rr_new = creal(dot(n, r, r));
        double beta = rr_new / rr;
        rr = rr_new;
        for (long k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
        ++it;
    }
    normal_op(L, U, kappa, (double *)Ap, xd, (double *)tmp);
    for (long k = 0; k < n; ++k) r[k] = b[k] - Ap[k];
    double relres = sqrt(creal(dot(n, r, r)) / bb);
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = relres;
    free(r);
    free(p);
    free(Ap);
    free(tmp);
    return relres <= tol ? 0 : 1;
}

/* ------------------------------------------------------------ threads -- */

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
