/*
 * sn_oracle.c -- plain, slow, FP64 reference of the DFEM S_n transport solve
 * of Tano & Ragusa, "Acceleration of Radiation Transport Solves Using
 * Artificial Neural Networks" (arXiv:1906.04017).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * reads this file; only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Equation numbers are the paper's, counted in order of appearance:
 *   (1) transport equation, (2) total source, (6)-(7) moment form,
 *   (3)-(5) Legendre expansion of the scattering and the addition theorem,
 *   (8)-(9) S_N discretisation, (10) inflow boundary condition,
 *   (11) DFEM trial expansion, (12) discrete DFEM system, (13) phi = D psi,
 *   (14) the per-cell system A psi = b, (21) source-iteration change.
 *
 * Readings of the paper taken here (where the text is silent or inconsistent):
 *   - Sec. 2 uses "+" for the inflow boundary (n.Omega < 0) when it defines
 *     the faces, but the per-cell system (14) puts the outflow matrix in A
 *     and the upwind matrix in b.  The oracle uses exactly that outflow form:
 *        A = sum_a Omega_a L_a + sum_{f: Omega.n_f > 0} (Omega.n_f) F_f + sigma_t M
 *        b = M S + sum_{f: Omega.n_f < 0} |Omega.n_f| F_f psi_up
 *     with L_a[k][j] = -int u_j d_a w_k (the Green's-theorem volume term of
 *     the streaming display in Sec. 2), F_f the face mass matrix and M the
 *     sigma_t-free mass matrix.
 *   - The scattering term of (12) multiplies the mass matrix without
 *     sigma_t (the integral written beside it has no sigma_t).
 *   - Trial space: tri-linear Q1 on axis-aligned boxes, 8 nodes, local node
 *     n = a + 2b + 4c (x fastest); the paper's "P_1" label is read as the
 *     8-node hexahedron it describes.
 *   - Quadrature: level-symmetric LQ_N (the paper leaves the set open).
 *   - Moments: sum of weights = 4 pi, phi = sum_d w_d psi_d, an isotropic
 *     source density is divided by 4 pi.
 *   - Groups: Jacobi source iteration (every group uses the previous phi).
 */
#include <math.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Gaussian elimination with partial pivoting (Sec. 2, after Eq. (14): the   */
/* per-cell system is "solved by direct Gauss Elimination").  Pivot = entry  */
/* of largest magnitude in the column, ties go to the lowest row.  A (n x n, */
/* row-major) and b are overwritten.  Returns 0, or -1 on a zero pivot.      */
/* ------------------------------------------------------------------------ */
int or_ge(int n, double *A, double *b, double *x)
{
    for (int col = 0; col < n; ++col) {
        int p = col;
        double best = fabs(A[col * n + col]);
        for (int r = col + 1; r < n; ++r) {
            double v = fabs(A[r * n + col]);
            if (v > best) { best = v; p = r; }
        }
        if (best == 0.0) return -1;
        if (p != col) {
            for (int c = 0; c < n; ++c) {
                double t = A[col * n + c]; A[col * n + c] = A[p * n + c]; A[p * n + c] = t;
            }
            double t = b[col]; b[col] = b[p]; b[p] = t;
        }
        for (int r = col + 1; r < n; ++r) {
            double l = A[r * n + col] / A[col * n + col];
            A[r * n + col] = 0.0;
            for (int c = col + 1; c < n; ++c) A[r * n + c] -= l * A[col * n + c];
            b[r] -= l * b[col];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int c = r + 1; c < n; ++c) s -= A[r * n + c] * x[c];
        x[r] = s / A[r * n + r];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Level-symmetric LQ_N quadrature (Sec. 2, Eqs. (8)-(9): the pairs          */
/* (Omega_d, w_d); the set itself is left open by the paper).                */
/* Per octant the N(N+2)/8 points are (mu_i, mu_j, mu_k) with i+j+k = N/2+2, */
/* mu_i^2 = mu_1^2 + (i-1) * 2 (1 - 3 mu_1^2) / (N - 2).  Points whose level */
/* triples are permutations of each other share a weight; the class weights  */
/* solve the even x-moment conditions sum w mu^(2m) = 1/(2m+1) for           */
/* m = 0, 2, 3, ..., K (K classes; m = 1 follows from symmetry).  mu_1 is    */
/* the standard LQ_N value.  Directions are ordered octant-major (octant bit */
/* 0: mu < 0, bit 1: eta < 0, bit 2: xi < 0), then i ascending, j ascending. */
/* Weights are scaled to sum to 4 pi.  Returns ndir, or -1 for an           */
/* unsupported order.                                                        */
/* ------------------------------------------------------------------------ */
int or_lqn(int N, double *omega, double *w)
{
    double mu1;
    switch (N) {
    case 2:  mu1 = 0.57735026918962576; break;
    case 4:  mu1 = 0.3500212; break;
    case 6:  mu1 = 0.2666355; break;
    case 8:  mu1 = 0.2182179; break;
    case 10: mu1 = 0.1893213; break;
    case 12: mu1 = 0.1672126; break;
    default: return -1;
    }
    int n2 = N / 2;
    double mu[8];
    for (int i = 0; i < n2; ++i) {
        double m2 = mu1 * mu1;
        if (N > 2) m2 += i * 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 2);
        mu[i] = sqrt(m2);
    }
    /* points of one octant and their classes */
    int lev[64][3], cls[64], ncls = 0, clsk[64][3], np = 0;
    for (int i = 1; i <= n2; ++i)
        for (int j = 1; j <= n2 + 1 - i; ++j) {
            int k = n2 + 2 - i - j;
            lev[np][0] = i; lev[np][1] = j; lev[np][2] = k;
            int s[3] = {i, j, k};
            for (int a = 0; a < 3; ++a)           /* sort the triple */
                for (int b2 = a + 1; b2 < 3; ++b2)
                    if (s[b2] < s[a]) { int t = s[a]; s[a] = s[b2]; s[b2] = t; }
            int c = -1;
            for (int q = 0; q < ncls; ++q)
                if (clsk[q][0] == s[0] && clsk[q][1] == s[1] && clsk[q][2] == s[2]) c = q;
            if (c < 0) { c = ncls++; clsk[c][0] = s[0]; clsk[c][1] = s[1]; clsk[c][2] = s[2]; }
            cls[np++] = c;
        }
    /* moment conditions */
    double A[64], b[8], x[8];
    for (int r = 0; r < ncls; ++r) {
        int m = (r == 0) ? 0 : r + 1;
        for (int c = 0; c < ncls; ++c) A[r * ncls + c] = 0.0;
        for (int p = 0; p < np; ++p) A[r * ncls + cls[p]] += pow(mu[lev[p][0] - 1], 2.0 * m);
        b[r] = 1.0 / (2.0 * m + 1.0);
    }
    if (or_ge(ncls, A, b, x) != 0) return -1;
    int d = 0;
    for (int o = 0; o < 8; ++o)
        for (int p = 0; p < np; ++p, ++d) {
            omega[3 * d + 0] = ((o & 1) ? -1.0 : 1.0) * mu[lev[p][0] - 1];
            omega[3 * d + 1] = ((o & 2) ? -1.0 : 1.0) * mu[lev[p][1] - 1];
            omega[3 * d + 2] = ((o & 4) ? -1.0 : 1.0) * mu[lev[p][2] - 1];
            w[d] = x[cls[p]] * (4.0 * PI / 8.0);
        }
    return d;
}

/* ------------------------------------------------------------------------ */
/* Element matrices on the box [0,dx]x[0,dy]x[0,dz] (Sec. 2, the streaming,  */
/* total-interaction and source displays before Eq. (12)), integrated with  */
/* 2x2x2 Gauss-Legendre points (exact for products of tri-linear functions). */
/*   M[k][j]    = int u_k u_j dV                                             */
/*   L[a][k][j] = -int u_j d_a u_k dV       (Green's-theorem volume term)    */
/*   G[a][k][j] = int u_k d_a u_j dV        (volume term before Green)       */
/*   F[f][k][j] = int_f u_k u_j dA, f = x-, x+, y-, y+, z-, z+               */
/* Basis u_n = beta_a(x) beta_b(y) beta_c(z), n = a + 2b + 4c,               */
/* beta_0(t) = 1 - t/h, beta_1(t) = t/h.                                     */
/* ------------------------------------------------------------------------ */
static double beta(int a, double t, double h) { return a ? t / h : 1.0 - t / h; }
static double dbeta(int a, double h) { return a ? 1.0 / h : -1.0 / h; }

static void basis(const double h[3], const double r[3], double u[8], double du[3][8])
{
    for (int n = 0; n < 8; ++n) {
        int ia[3] = {n & 1, (n >> 1) & 1, (n >> 2) & 1};
        double v[3], dv[3];
        for (int ax = 0; ax < 3; ++ax) { v[ax] = beta(ia[ax], r[ax], h[ax]); dv[ax] = dbeta(ia[ax], h[ax]); }
        u[n] = v[0] * v[1] * v[2];
        du[0][n] = dv[0] * v[1] * v[2];
        du[1][n] = v[0] * dv[1] * v[2];
        du[2][n] = v[0] * v[1] * dv[2];
    }
}

void or_element(double dx, double dy, double dz, double *M, double *L, double *G, double *F)
{
    const double h[3] = {dx, dy, dz};
    const double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
    memset(M, 0, 64 * sizeof(double));
    memset(L, 0, 3 * 64 * sizeof(double));
    memset(G, 0, 3 * 64 * sizeof(double));
    memset(F, 0, 6 * 64 * sizeof(double));
    /* volume terms */
    for (int p0 = 0; p0 < 2; ++p0)
        for (int p1 = 0; p1 < 2; ++p1)
            for (int p2 = 0; p2 < 2; ++p2) {
                double r[3] = {gp[p0] * dx, gp[p1] * dy, gp[p2] * dz};
                double wt = 0.125 * dx * dy * dz;
                double u[8], du[3][8];
                basis(h, r, u, du);
                for (int k = 0; k < 8; ++k)
                    for (int j = 0; j < 8; ++j) {
                        M[k * 8 + j] += wt * u[k] * u[j];
                        for (int ax = 0; ax < 3; ++ax) {
                            L[ax * 64 + k * 8 + j] -= wt * u[j] * du[ax][k];
                            G[ax * 64 + k * 8 + j] += wt * u[k] * du[ax][j];
                        }
                    }
            }
    /* face terms: face f = 2*axis + side, side 0 at coordinate 0, side 1 at h */
    for (int f = 0; f < 6; ++f) {
        int ax = f / 2, side = f % 2;
        int t1 = (ax + 1) % 3, t2 = (ax + 2) % 3;
        for (int p1 = 0; p1 < 2; ++p1)
            for (int p2 = 0; p2 < 2; ++p2) {
                double r[3];
                r[ax] = side ? h[ax] : 0.0;
                r[t1] = gp[p1] * h[t1];
                r[t2] = gp[p2] * h[t2];
                double wt = 0.25 * h[t1] * h[t2];
                double u[8], du[3][8];
                basis(h, r, u, du);
                for (int k = 0; k < 8; ++k)
                    for (int j = 0; j < 8; ++j) F[f * 64 + k * 8 + j] += wt * u[k] * u[j];
            }
    }
}

/* Outward normal component of face f along its axis. */
static double face_sign(int f) { return (f % 2) ? 1.0 : -1.0; }

/* Local node on face f of a cell with in-face index t (0..3).  For an x-face */
/* t = b + 2c, for a y-face t = a + 2c, for a z-face t = a + 2b.             */
static int face_node(int f, int t)
{
    int ax = f / 2, side = f % 2;
    int lo = t & 1, hi = (t >> 1) & 1;
    int a, b, c;
    if (ax == 0) { a = side; b = lo; c = hi; }
    else if (ax == 1) { a = lo; b = side; c = hi; }
    else { a = lo; b = hi; c = side; }
    return a + 2 * b + 4 * c;
}

/* ------------------------------------------------------------------------ */
/* Per-cell system (14) in the outflow form (see the header).  up[12] holds  */
/* the upwind face values on the inflow face of each axis: x-face (4), then  */
/* y-face (4), then z-face (4), in-face order as in face_node().  Omega_a = 0 */
/* means no flow through that axis' faces.                                   */
/* ------------------------------------------------------------------------ */
typedef struct { double M[64], L[192], G[192], F[384]; } or_elem;

static void assemble(const or_elem *e, const double om[3], double sigt,
                     const double S[8], const double up[12], double A[64], double b[8])
{
    for (int i = 0; i < 64; ++i)
        A[i] = om[0] * e->L[i] + om[1] * e->L[64 + i] + om[2] * e->L[128 + i] + sigt * e->M[i];
    for (int k = 0; k < 8; ++k) {
        double s = 0.0;
        for (int j = 0; j < 8; ++j) s += e->M[k * 8 + j] * S[j];
        b[k] = s;
    }
    for (int ax = 0; ax < 3; ++ax) {
        if (om[ax] == 0.0) continue;
        int fout = 2 * ax + (om[ax] > 0.0 ? 1 : 0);
        int fin = 2 * ax + (om[ax] > 0.0 ? 0 : 1);
        double on_out = om[ax] * face_sign(fout);          /* > 0 */
        double on_in = fabs(om[ax] * face_sign(fin));      /* |Omega.n| on inflow */
        for (int i = 0; i < 64; ++i) A[i] += on_out * e->F[fout * 64 + i];
        double ext[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int t = 0; t < 4; ++t) ext[face_node(fin, t)] = up[4 * ax + t];
        for (int k = 0; k < 8; ++k) {
            double s = 0.0;
            for (int j = 0; j < 8; ++j) s += e->F[fin * 64 + k * 8 + j] * ext[j];
            b[k] += on_in * s;
        }
    }
}

/* Exported for the tests: the outflow form above and the inflow form that  */
/* Green's theorem turns it into (A = sum Omega_a G_a + sum_inflow |Omega.n| */
/* F_f + sigma_t M).  The two must agree to round-off.                       */
void or_assemble(double dx, double dy, double dz, const double om[3], double sigt,
                 const double S[8], const double up[12], double *A, double *b)
{
    or_elem e;
    or_element(dx, dy, dz, e.M, e.L, e.G, e.F);
    assemble(&e, om, sigt, S, up, A, b);
}

void or_assemble_inflow_form(double dx, double dy, double dz, const double om[3], double sigt, double *A)
{
    or_elem e;
    or_element(dx, dy, dz, e.M, e.L, e.G, e.F);
    for (int i = 0; i < 64; ++i)
        A[i] = om[0] * e.G[i] + om[1] * e.G[64 + i] + om[2] * e.G[128 + i] + sigt * e.M[i];
    for (int ax = 0; ax < 3; ++ax) {
        if (om[ax] == 0.0) continue;
        int fin = 2 * ax + (om[ax] > 0.0 ? 0 : 1);
        for (int i = 0; i < 64; ++i) A[i] += fabs(om[ax]) * e.F[fin * 64 + i];
    }
}

/* One-cell problem: in27 = Omega(3), (dx,dy,dz), sigma_t, S(8), up(12).     */
/* Assemble (14) and solve it by Gaussian elimination.                       */
int or_cell_solve(const double *in27, double *psi)
{
    or_elem e;
    double A[64], b[8];
    or_element(in27[3], in27[4], in27[5], e.M, e.L, e.G, e.F);
    assemble(&e, in27, in27[6], in27 + 7, in27 + 15, A, b);
    return or_ge(8, A, b, psi);
}

int or_cell_solve_batch(long n, const double *in27, double *psi)
{
    int bad = 0;
    for (long i = 0; i < n; ++i)
        if (or_cell_solve(in27 + 27 * i, psi + 8 * i) != 0) bad = 1;
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* The paper's per-octant networks as a one-cell solver (Sec. 3, Eqs. (15)-  */
/* (18); Sec. 4: one network per octant).  Network o serves the directions   */
/* with octant bits (mu < 0) | (eta < 0) << 1 | (xi < 0) << 2.  Inputs, in   */
/* the order of the list in Sec. 3: the 12 upwind face values, mu, eta, the  */
/* 8 nodal sources, sigma_t, dx, dy, dz; each scaled by Eq. (16),            */
/* x = (I - alpha (I_min + I_max) / 2) / |I_max - I_min|, alpha = 0.27.       */
/* h = tanh(W1 x + b1); psi_d = z_d (z_d >= 0) or beta (e^{z_d} - 1) with     */
/* z = W2 h + b2 and beta = 0.1 max |psi_inc| over the 12 upwind values.      */
/* Parameters per octant (288): W1[8][26], b1[8], W2[8][8], b2[8].           */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double *p;      /* [8][288]                                       */
    const double *lo;     /* [8][26] a-priori input minima                   */
    const double *hi;     /* [8][26] a-priori input maxima                   */
} or_octnet;

void or_octnet_cell(const or_octnet *net, const double *in27, double *psi)
{
    const int o = (in27[0] < 0.0) | ((in27[1] < 0.0) << 1) | ((in27[2] < 0.0) << 2);
    const double *P = net->p + 288 * o, *lo = net->lo + 26 * o, *hi = net->hi + 26 * o;
    const double *W1 = P, *b1 = P + 208, *W2 = P + 216, *b2 = P + 280;
    double I[26], x[26], h[8];
    for (int t = 0; t < 12; ++t) I[t] = in27[15 + t];
    I[12] = in27[0];
    I[13] = in27[1];
    for (int n = 0; n < 8; ++n) I[14 + n] = in27[7 + n];
    I[22] = in27[6];
    for (int a = 0; a < 3; ++a) I[23 + a] = in27[3 + a];
    for (int j = 0; j < 26; ++j) x[j] = (I[j] - 0.27 * 0.5 * (lo[j] + hi[j])) / fabs(hi[j] - lo[j]);
    double bm = 0.0;
    for (int t = 0; t < 12; ++t) bm = fmax(bm, fabs(in27[15 + t]));
    const double beta = 0.1 * bm;
    for (int k = 0; k < 8; ++k) {
        double a = b1[k];
        for (int j = 0; j < 26; ++j) a += W1[26 * k + j] * x[j];
        h[k] = tanh(a);
    }
    for (int d = 0; d < 8; ++d) {
        double z = b2[d];
        for (int k = 0; k < 8; ++k) z += W2[8 * d + k] * h[k];
        psi[d] = z >= 0.0 ? z : beta * expm1(z);
    }
}

void or_octnet_cell_batch(const or_octnet *net, long n, const double *in27, double *psi)
{
    for (long i = 0; i < n; ++i) or_octnet_cell(net, in27 + 27 * i, psi + 8 * i);
}

/* ------------------------------------------------------------------------ */
/* The workload's surrogate network as a one-cell solver: 27 inputs -> 64    */
/* ReLU -> 8 linear outputs (one hidden layer, Eq. (15)), one network for    */
/* every octant through the mirror symmetry of the DFEM system.  The input   */
/* construction (the counterpart of the scaling of Eq. (16)) follows the     */
/* Python oracle (oracle/mlp.py) term by term:                               */
/*   mirror into the positive octant: node k of the canonical cell is node   */
/*   k ^ m, m = (mu<0) | (eta<0)<<1 | (xi<0)<<2, in-face t of the x-face is   */
/*   t ^ ((eta<0) | (xi<0)<<1) (y-, z-faces alike);                          */
/*   s = max(max |S_c|, max |up_c|), 1/s taken as 0 for s <= 1e-30;          */
/*   x = [2|Omega| - 1, (log h + 1.15) / 1.15, log(max(sigma_t, 1e-6)) / 4.5, */
/*        S_c / s, up_c / s];                                                */
/*   psi (physical node k) = s * o[k ^ m].                                    */
/* With bf16 set, the rounding steps of the tensor-core path are applied:    */
/* the one-cell inputs and the parameters to FP32, the features, W1, W2 and  */
/* the hidden activations to BF16 (round to nearest, ties to even), sums and */
/* biases otherwise exact.  Parameters (2312): W1[64][27], b1[64], W2[8][64], */
/* b2[8].                                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double *p;
    int bf16;
} or_mlp;

static double to_f32(double v) { return (double)(float)v; }

static double to_bf16(double v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    uint64_t w = u;
    w = ((w + 0x7FFFu + ((w >> 16) & 1u)) >> 16) << 16;
    u = (uint32_t)w;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* parameters as the network uses them: rounded to FP32, W1 and W2 further to */
/* BF16, when bf16 is set; unchanged otherwise                                */
static void mlp_params(const or_mlp *net, double *q)
{
    for (int i = 0; i < 2312; ++i) {
        const int is_w = i < 64 * 27 || (i >= 64 * 27 + 64 && i < 64 * 27 + 64 + 8 * 64);
        q[i] = !net->bf16 ? net->p[i] : (is_w ? to_bf16(to_f32(net->p[i])) : to_f32(net->p[i]));
    }
}

/* one cell with the parameters q of mlp_params */
static void mlp_cell(const double *q, int rb, const double *in27_, double *psi)
{
    double in27[27];
    for (int i = 0; i < 27; ++i) in27[i] = rb ? to_f32(in27_[i]) : in27_[i];
    const int fx = in27[0] < 0.0, fy = in27[1] < 0.0, fz = in27[2] < 0.0;
    const int m = fx | (fy << 1) | (fz << 2);
    double Sc[8], Uc[12];
    for (int k = 0; k < 8; ++k) Sc[k] = in27[7 + (k ^ m)];
    for (int t = 0; t < 4; ++t) {
        Uc[t] = in27[15 + (t ^ (fy | (fz << 1)))];
        Uc[4 + t] = in27[19 + (t ^ (fx | (fz << 1)))];
        Uc[8 + t] = in27[23 + (t ^ (fx | (fy << 1)))];
    }
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s = fmax(s, fabs(Sc[k]));
    for (int t = 0; t < 12; ++t) s = fmax(s, fabs(Uc[t]));
    const double inv = s > 1e-30 ? 1.0 / s : 0.0;
    double x[27];
    for (int a = 0; a < 3; ++a) {
        x[a] = 2.0 * fabs(in27[a]) - 1.0;
        x[3 + a] = (log(in27[3 + a]) + 1.15) / 1.15;
    }
    x[6] = log(fmax(in27[6], 1e-6)) / 4.5;
    for (int k = 0; k < 8; ++k) x[7 + k] = Sc[k] * inv;
    for (int t = 0; t < 12; ++t) x[15 + t] = Uc[t] * inv;
    if (rb)
        for (int i = 0; i < 27; ++i) x[i] = to_bf16(x[i]);
    const double *W1 = q, *b1 = W1 + 64 * 27, *W2 = b1 + 64, *b2 = W2 + 8 * 64;
    double h[64], o[8];
    for (int j = 0; j < 64; ++j) {
        double a = b1[j];
        for (int i = 0; i < 27; ++i) a += W1[27 * j + i] * x[i];
        h[j] = a > 0.0 ? a : 0.0;
        if (rb) h[j] = to_bf16(h[j]);
    }
    for (int d = 0; d < 8; ++d) {
        double z = b2[d];
        for (int j = 0; j < 64; ++j) z += W2[64 * d + j] * h[j];
        o[d] = z;
    }
    for (int k = 0; k < 8; ++k) psi[k] = s * o[k ^ m];
}

void or_mlp_cell_batch(const or_mlp *net, long n, const double *in27, double *psi)
{
    double q[2312];
    mlp_params(net, q);
    for (long i = 0; i < n; ++i) mlp_cell(q, net->bf16, in27 + 27 * i, psi + 8 * i);
}

/* a one-cell solver handed to the sweep in place of assembly and elimination */
typedef struct {
    void (*cell)(const void *ctx, const double *in27, double *psi);
    const void *ctx;
} or_cellnet;

static void octnet_cb(const void *ctx, const double *in27, double *psi)
{
    or_octnet_cell((const or_octnet *)ctx, in27, psi);
}

/* the surrogate prepared for a sweep: its parameters as used, and the mode */
typedef struct {
    double q[2312];
    int bf16;
} or_mlp_prepared;

static void mlp_cb(const void *ctx, const double *in27, double *psi)
{
    const or_mlp_prepared *m = (const or_mlp_prepared *)ctx;
    mlp_cell(m->q, m->bf16, in27, psi);
}

/* ------------------------------------------------------------------------ */
/* General hexahedral cells (the shape change of the cells of Sec. 2's       */
/* closing remarks): a trilinear map x(xi) = sum_n X_n N_n(xi) of the unit   */
/* cube, N_n = prod over the axes of xi_a or 1 - xi_a by the bits of          */
/* n = a + 2b + 4c, the same N_n as trial and test functions (isoparametric  */
/* Q1).  Element matrices:                                                   */
/*   M[k][j]       = int N_k N_j dV                                          */
/*   L_a[k][j]     = -int N_j d_a N_k dV                                     */
/*   Fv[f][a][k][j] = int_f n_a N_k N_j dS  (outward area vector of face f)  */
/* With dV = det J dxi and d_a N = sum_s adj(J)[s][a] d_s N / det J, every     */
/* integrand (det J N N, adj(J) terms, the face area vectors) is a            */
/* polynomial of degree <= 4 per axis, so 3-point Gauss quadrature per axis  */
/* integrates them exactly.  Face f = 2a + side (side 1: xi_a = 1); the face  */
/* area vector is +-(dx/dxi_p x dx/dxi_q) with (a, p, q) cyclic, + on side 1. */
/* The per-cell system is the outflow form of (14) with the faces' Omega.n   */
/* taken from Fv; the mesh keeps the structured topology, and a face is      */
/* inflow or outflow for a direction by the sign of Omega_a as for a box    */
/* (meshes where Omega.n changes sign on a face are outside this reading).  */
/* ------------------------------------------------------------------------ */
typedef struct { double M[64], L[3][64], Fv[6][3][64]; } or_hex;

static void hex_shape(const double xi[3], double N[8], double dN[8][3])
{
    for (int n = 0; n < 8; ++n) {
        double f[3], df[3];
        for (int a = 0; a < 3; ++a) {
            const int bit = (n >> a) & 1;
            f[a] = bit ? xi[a] : 1.0 - xi[a];
            df[a] = bit ? 1.0 : -1.0;
        }
        N[n] = f[0] * f[1] * f[2];
        dN[n][0] = df[0] * f[1] * f[2];
        dN[n][1] = f[0] * df[1] * f[2];
        dN[n][2] = f[0] * f[1] * df[2];
    }
}

void or_hex_element(const double *X /* [8][3] */, or_hex *e)
{
    const double g[3] = {0.5 - 0.5 * sqrt(0.6), 0.5, 0.5 + 0.5 * sqrt(0.6)};
    const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    memset(e, 0, sizeof(*e));
    for (int i0 = 0; i0 < 3; ++i0)
        for (int i1 = 0; i1 < 3; ++i1)
            for (int i2 = 0; i2 < 3; ++i2) {
                const double xi[3] = {g[i0], g[i1], g[i2]};
                const double w = gw[i0] * gw[i1] * gw[i2];
                double N[8], dN[8][3], J[3][3] = {{0}};
                hex_shape(xi, N, dN);
                for (int n = 0; n < 8; ++n)
                    for (int r = 0; r < 3; ++r)
                        for (int c = 0; c < 3; ++c) J[r][c] += X[3 * n + r] * dN[n][c];
                /* adj(J)[s][a]: the cofactor transpose, J adj(J) = det J I */
                double adj[3][3];
                adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
                adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
                adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
                adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
                adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
                adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
                adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
                adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
                adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
                const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
                for (int k = 0; k < 8; ++k)
                    for (int j = 0; j < 8; ++j) {
                        e->M[8 * k + j] += w * det * N[k] * N[j];
                        for (int a = 0; a < 3; ++a) {
                            double dk = 0.0;   /* det J * d_a N_k */
                            for (int s2 = 0; s2 < 3; ++s2) dk += adj[s2][a] * dN[k][s2];
                            e->L[a][8 * k + j] -= w * N[j] * dk;
                        }
                    }
            }
    for (int f = 0; f < 6; ++f) {
        const int a = f / 2, side = f % 2, p = (a + 1) % 3, q = (a + 2) % 3;
        for (int ip = 0; ip < 3; ++ip)
            for (int iq = 0; iq < 3; ++iq) {
                double xi[3];
                xi[a] = side;
                xi[p] = g[ip];
                xi[q] = g[iq];
                const double w = gw[ip] * gw[iq];
                double N[8], dN[8][3], tp[3] = {0, 0, 0}, tq[3] = {0, 0, 0};
                hex_shape(xi, N, dN);
                for (int n = 0; n < 8; ++n)
                    for (int r = 0; r < 3; ++r) {
                        tp[r] += X[3 * n + r] * dN[n][p];
                        tq[r] += X[3 * n + r] * dN[n][q];
                    }
                double av[3] = {tp[1] * tq[2] - tp[2] * tq[1], tp[2] * tq[0] - tp[0] * tq[2],
                                tp[0] * tq[1] - tp[1] * tq[0]};
                const double sg = side ? 1.0 : -1.0;
                for (int k = 0; k < 8; ++k)
                    for (int j = 0; j < 8; ++j)
                        for (int c = 0; c < 3; ++c) e->Fv[f][c][8 * k + j] += w * sg * av[c] * N[k] * N[j];
            }
    }
}

/* Elements of every cell of a structured mesh with vertex coordinates         */
/* xyz [(nx+1)(ny+1)(nz+1)][3], vertex (i,j,k) at i + (nx+1)(j + (ny+1) k).     */
void or_hex_elements(int nx, int ny, int nz, const double *xyz, or_hex *out)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double X[24];
                for (int n = 0; n < 8; ++n) {
                    const long v = (i + (n & 1)) + (long)(nx + 1) * ((j + ((n >> 1) & 1)) + (long)(ny + 1) * (k + (n >> 2)));
                    for (int r = 0; r < 3; ++r) X[3 * n + r] = xyz[3 * v + r];
                }
                or_hex_element(X, out + i + (long)nx * (j + (long)ny * k));
            }
}

/* Outflow form of (14) on a general cell: A = sum_a Omega_a L_a + sigma_t M  */
/* + sum over outflow faces of Omega.Fv; b = M S + sum over inflow faces of   */
/* (-Omega.Fv) applied to the upwind values on that face.                      */
static void assemble_hex(const or_hex *e, const double om[3], double sigt, const double S[8],
                         const double up[12], double A[64], double b[8])
{
    for (int i = 0; i < 64; ++i)
        A[i] = om[0] * e->L[0][i] + om[1] * e->L[1][i] + om[2] * e->L[2][i] + sigt * e->M[i];
    for (int k = 0; k < 8; ++k) {
        double s = 0.0;
        for (int j = 0; j < 8; ++j) s += e->M[8 * k + j] * S[j];
        b[k] = s;
    }
    for (int ax = 0; ax < 3; ++ax) {
        if (om[ax] == 0.0) continue;
        const int fout = 2 * ax + (om[ax] > 0.0 ? 1 : 0), fin = 2 * ax + (om[ax] > 0.0 ? 0 : 1);
        for (int i = 0; i < 64; ++i)
            A[i] += om[0] * e->Fv[fout][0][i] + om[1] * e->Fv[fout][1][i] + om[2] * e->Fv[fout][2][i];
        double ext[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int t = 0; t < 4; ++t) ext[face_node(fin, t)] = up[4 * ax + t];
        for (int k = 0; k < 8; ++k) {
            double s = 0.0;
            for (int j = 0; j < 8; ++j)
                s -= (om[0] * e->Fv[fin][0][8 * k + j] + om[1] * e->Fv[fin][1][8 * k + j] +
                      om[2] * e->Fv[fin][2][8 * k + j]) * ext[j];
            b[k] += s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Problem description.                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    int ndir;
    const double *omega;    /* [ndir][3]                                    */
    const double *w;        /* [ndir], sum 4 pi                             */
    int G;
    const double *sigt;     /* [G][ncell] total cross section               */
    const double *sigs;     /* [G][ncell] scattering out of group g         */
    const double *q;        /* [G][ncell] isotropic emission density        */
    const double *xfer;     /* [G][G] fraction of g' scattering into g      */
    const double *psi_inc;  /* [G][6] isotropic inflow on x-,x+,y-,y+,z-,z+ */
    const void *hex;        /* NULL: box cells dx x dy x dz; else or_hex [ncell] */
} or_problem;

static long ncell_of(const or_problem *p) { return (long)p->nx * p->ny * p->nz; }

/* ------------------------------------------------------------------------ */
/* Sweep of one direction and group (Sec. 2, after Eq. (14): start at the    */
/* cells whose inflow is known, move to downstream neighbours).  Cells are   */
/* visited in upwind lexicographic order.  S is the nodal source density     */
/* [ncell][8] for this direction.  Boundary inflow comes from bnd_{x,y,z}    */
/* (per-face nodal values, layout [j + ny k][4], [i + nx k][4], [i + nx j][4]) */
/* or, when a pointer is NULL, from the problem's constant psi_inc (Eq. (10)) */
/* for group g.  tallies[0..3] += leakage, collision, source, inflow.        */
/* ------------------------------------------------------------------------ */
static int sweep_dir(const or_problem *p, const or_elem *e, const or_cellnet *net, int d, int g,
                     const double *S, const double *bx, const double *by, const double *bz, double *psi,
                     double tal[4])
{
    const double *om = p->omega + 3 * d;
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const long nc = ncell_of(p);
    int fin[3], fout[3];
    for (int ax = 0; ax < 3; ++ax) {
        fin[ax] = 2 * ax + (om[ax] >= 0.0 ? 0 : 1);
        fout[ax] = 2 * ax + (om[ax] >= 0.0 ? 1 : 0);
    }
    /* face integral weights: int_f u_j over face f = column sums of F_f */
    double fint[6][8];
    for (int f = 0; f < 6; ++f)
        for (int j = 0; j < 8; ++j) {
            double s = 0.0;
            for (int k = 0; k < 8; ++k) s += e->F[f * 64 + k * 8 + j];
            fint[f][j] = s;
        }
    double vint[8];
    for (int j = 0; j < 8; ++j) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += e->M[k * 8 + j];
        vint[j] = s;
    }
    for (int kk = 0; kk < nz; ++kk) {
        int k = om[2] >= 0.0 ? kk : nz - 1 - kk;
        for (int jj = 0; jj < ny; ++jj) {
            int j = om[1] >= 0.0 ? jj : ny - 1 - jj;
            for (int ii = 0; ii < nx; ++ii) {
                int i = om[0] >= 0.0 ? ii : nx - 1 - ii;
                long c = i + (long)nx * (j + (long)ny * k);
                double up[12];
                int onbnd[3];
                for (int ax = 0; ax < 3; ++ax) {
                    int idx[3] = {i, j, k}, n[3] = {nx, ny, nz};
                    int ui = idx[ax] + (om[ax] >= 0.0 ? -1 : 1);
                    onbnd[ax] = (ui < 0 || ui >= n[ax]);
                    for (int t = 0; t < 4; ++t) {
                        if (!onbnd[ax]) {
                            int nb[3] = {i, j, k};
                            nb[ax] = ui;
                            long cu = nb[0] + (long)nx * (nb[1] + (long)ny * nb[2]);
                            /* the upwind cell's node on its outflow face (the */
                            /* face opposite to our inflow face, same in-face t) */
                            up[4 * ax + t] = psi[8 * cu + face_node(fout[ax], t)];
                        } else {
                            const double *bv = ax == 0 ? bx : (ax == 1 ? by : bz);
                            if (bv) {
                                long fi = ax == 0 ? j + (long)ny * k : (ax == 1 ? i + (long)nx * k : i + (long)nx * j);
                                up[4 * ax + t] = bv[4 * fi + t];
                            } else {
                                up[4 * ax + t] = p->psi_inc[6 * g + fin[ax]];
                            }
                        }
                    }
                }
                double x[8];
                if (net) {
                    /* the cell's one-cell problem handed to the network */
                    double in27[27];
                    for (int a = 0; a < 3; ++a) in27[a] = om[a];
                    in27[3] = p->dx; in27[4] = p->dy; in27[5] = p->dz;
                    in27[6] = p->sigt[(long)g * nc + c];
                    for (int n = 0; n < 8; ++n) in27[7 + n] = S[8 * c + n];
                    for (int t = 0; t < 12; ++t) in27[15 + t] = up[t];
                    net->cell(net->ctx, in27, x);
                } else if (p->hex) {
                    double A[64], b[8];
                    assemble_hex((const or_hex *)p->hex + c, om, p->sigt[(long)g * nc + c], S + 8 * c, up, A, b);
                    if (or_ge(8, A, b, x) != 0) return -1;
                } else {
                    double A[64], b[8];
                    assemble(e, om, p->sigt[(long)g * nc + c], S + 8 * c, up, A, b);
                    if (or_ge(8, A, b, x) != 0) return -1;
                }
                for (int n = 0; n < 8; ++n) psi[8 * c + n] = x[n];
                if (tal && p->hex) {
                    /* the same tallies from the cell's own matrices: w = 1 = sum of */
                    /* the test functions, so row sums give the face and volume     */
                    /* integrals of psi                                              */
                    const or_hex *h = (const or_hex *)p->hex + c;
                    for (int ax = 0; ax < 3; ++ax) {
                        if (om[ax] == 0.0) continue;
                        int idx[3] = {i, j, k}, n[3] = {nx, ny, nz};
                        int di = idx[ax] + (om[ax] >= 0.0 ? 1 : -1);
                        for (int jn = 0; jn < 8; ++jn) {
                            double fo = 0.0, fi = 0.0;
                            for (int kn = 0; kn < 8; ++kn)
                                for (int cc = 0; cc < 3; ++cc) {
                                    fo += om[cc] * h->Fv[fout[ax]][cc][8 * kn + jn];
                                    fi -= om[cc] * h->Fv[fin[ax]][cc][8 * kn + jn];
                                }
                            if (di < 0 || di >= n[ax]) tal[0] += fo * x[jn];
                            if (onbnd[ax]) {
                                for (int t = 0; t < 4; ++t)
                                    if (face_node(fin[ax], t) == jn) tal[3] += fi * up[4 * ax + t];
                            }
                        }
                    }
                    double sc = 0.0, ss = 0.0;
                    for (int jn = 0; jn < 8; ++jn) {
                        double v = 0.0;
                        for (int kn = 0; kn < 8; ++kn) v += h->M[8 * kn + jn];
                        sc += v * x[jn];
                        ss += v * S[8 * c + jn];
                    }
                    tal[1] += p->sigt[(long)g * nc + c] * sc;
                    tal[2] += ss;
                } else if (tal) {
                    for (int ax = 0; ax < 3; ++ax) {
                        if (om[ax] == 0.0) continue;
                        int idx[3] = {i, j, k}, n[3] = {nx, ny, nz};
                        int di = idx[ax] + (om[ax] >= 0.0 ? 1 : -1);
                        if (di < 0 || di >= n[ax]) {          /* boundary outflow */
                            double s = 0.0;
                            for (int jn = 0; jn < 8; ++jn) s += fint[fout[ax]][jn] * x[jn];
                            tal[0] += fabs(om[ax]) * s;
                        }
                        if (onbnd[ax]) {                        /* boundary inflow */
                            double s = 0.0;
                            for (int t = 0; t < 4; ++t) s += fint[fin[ax]][face_node(fin[ax], t)] * up[4 * ax + t];
                            tal[3] += fabs(om[ax]) * s;
                        }
                    }
                    double sc = 0.0, ss = 0.0;
                    for (int jn = 0; jn < 8; ++jn) { sc += vint[jn] * x[jn]; ss += vint[jn] * S[8 * c + jn]; }
                    tal[1] += p->sigt[(long)g * nc + c] * sc;
                    tal[2] += ss;
                }
            }
        }
    }
    return 0;
}

int or_sweep_dir(const or_problem *p, int d, int g, const double *S, const double *bx,
                 const double *by, const double *bz, double *psi, double *tal)
{
    or_elem e;
    or_element(p->dx, p->dy, p->dz, e.M, e.L, e.G, e.F);
    return sweep_dir(p, &e, NULL, d, g, S, bx, by, bz, psi, tal);
}

/* ------------------------------------------------------------------------ */
/* Full sweep for groups [g0,g1) and directions [d0,d1) with the isotropic   */
/* per-group source S[g][cell][8]; phi[g][cell][8] = sum_d w_d psi_d          */
/* (Eq. (9) with Y_00 absorbed in the 4 pi normalisation, Eq. (13)).         */
/* Groups run in parallel (each group's phi is summed over directions in a   */
/* fixed order, so the result does not depend on the thread count).          */
/* tal[4] receives the weighted balance tallies.  Returns 0 or -1.           */
/* ------------------------------------------------------------------------ */
static int sweep_range(const or_problem *p, const or_cellnet *net, const double *S, double *phi, int g0, int g1,
                       int d0, int d1, double *tal)
{
    or_elem e;
    or_element(p->dx, p->dy, p->dz, e.M, e.L, e.G, e.F);
    const long nc = ncell_of(p);
    int bad = 0;
    double gt[64][4];
    memset(gt, 0, sizeof(gt));
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int g = g0; g < g1; ++g) {
        double *psi = (double *)malloc(sizeof(double) * 8 * nc);
        double *ph = phi + (long)g * nc * 8;
        for (long i = 0; i < 8 * nc; ++i) ph[i] = 0.0;
        for (int d = d0; d < d1; ++d) {
            double t[4] = {0, 0, 0, 0};
            if (sweep_dir(p, &e, net, d, g, S + (long)g * nc * 8, NULL, NULL, NULL, psi, t) != 0) bad = 1;
            for (long i = 0; i < 8 * nc; ++i) ph[i] += p->w[d] * psi[i];
            for (int m = 0; m < 4; ++m) gt[g][m] += p->w[d] * t[m];
        }
        free(psi);
    }
    if (tal)
        for (int g = g0; g < g1; ++g)
            for (int m = 0; m < 4; ++m) tal[m] += gt[g][m];
    return bad ? -1 : 0;
}

int or_sweep(const or_problem *p, const double *S, double *phi, int g0, int g1, int d0, int d1, double *tal)
{
    return sweep_range(p, NULL, S, phi, g0, g1, d0, d1, tal);
}

/* The same sweep with every per-cell solve replaced by the octant networks */
/* (Sec. 4: the assembly and solve of (14) give way to building the input   */
/* vector and one evaluation of the network).                               */
int or_sweep_octnet(const or_problem *p, const or_octnet *net, const double *S, double *phi, int g0, int g1,
                    int d0, int d1, double *tal)
{
    const or_cellnet cn = {octnet_cb, net};
    return sweep_range(p, &cn, S, phi, g0, g1, d0, d1, tal);
}

/* The same with the workload's surrogate network as the cell solver.      */
int or_sweep_mlp(const or_problem *p, const or_mlp *net, const double *S, double *phi, int g0, int g1, int d0,
                 int d1, double *tal)
{
    or_mlp_prepared *m = (or_mlp_prepared *)malloc(sizeof(or_mlp_prepared));
    if (!m) return -1;
    mlp_params(net, m->q);
    m->bf16 = net->bf16;
    const or_cellnet cn = {mlp_cb, m};
    const int rc = sweep_range(p, &cn, S, phi, g0, g1, d0, d1, tal);
    free(m);
    return rc;
}

/* The same with the residual gate of the surrogate form: the network's     */
/* prediction psi of a cell is kept when ||b - A psi||_2 <= tau ||b||_2 for */
/* the cell's own system (14) (FP64, assembled as above), else the cell is */
/* solved by elimination.  *fallbacks (may be NULL) receives the number of */
/* cells sent to elimination.  tau = 0 gives or_sweep's flux, a tau above  */
/* every residual or_sweep_mlp's.                                          */
typedef struct {
    or_mlp_prepared m;
    or_elem e;
    double tau;
    long fallbacks;
} or_mlp_gated;

static void mlp_gated_cb(const void *ctx, const double *in27, double *psi)
{
    or_mlp_gated *m = (or_mlp_gated *)ctx;
    mlp_cell(m->m.q, m->m.bf16, in27, psi);
    double A[64], b[8];
    assemble(&m->e, in27, in27[6], in27 + 7, in27 + 15, A, b);
    double rr = 0.0, bb = 0.0;
    for (int k = 0; k < 8; ++k) {
        double r = b[k];
        for (int j = 0; j < 8; ++j) r -= A[8 * k + j] * psi[j];
        rr += r * r;
        bb += b[k] * b[k];
    }
    if (!(rr <= m->tau * m->tau * bb)) {
        double x[8];
        if (or_ge(8, A, b, x) == 0)
            for (int k = 0; k < 8; ++k) psi[k] = x[k];
        else
            for (int k = 0; k < 8; ++k) psi[k] = NAN;
#pragma omp atomic
        m->fallbacks += 1;
    }
}

int or_sweep_mlp_gated(const or_problem *p, const or_mlp *net, double tau, const double *S, double *phi, int g0,
                       int g1, int d0, int d1, double *tal, long *fallbacks)
{
    or_mlp_gated *m = (or_mlp_gated *)malloc(sizeof(or_mlp_gated));
    if (!m) return -1;
    mlp_params(net, m->m.q);
    m->m.bf16 = net->bf16;
    or_element(p->dx, p->dy, p->dz, m->e.M, m->e.L, m->e.G, m->e.F);
    m->tau = tau;
    m->fallbacks = 0;
    const or_cellnet cn = {mlp_gated_cb, m};
    const int rc = sweep_range(p, &cn, S, phi, g0, g1, d0, d1, tal);
    if (fallbacks) *fallbacks = m->fallbacks;
    free(m);
    return rc;
}

/* Isotropic source build (Eqs. (2), (6) with the P_0 term only):           */
/* S_g = (sum_g' xfer[g'][g] sigs_g' phi_g' + q_g) / (4 pi), nodal.           */
void or_source(const or_problem *p, const double *phi, double *S)
{
    const long nc = ncell_of(p);
    for (int g = 0; g < p->G; ++g)
        for (long c = 0; c < nc; ++c)
            for (int n = 0; n < 8; ++n) {
                double s = p->q[(long)g * nc + c];
                for (int gp = 0; gp < p->G; ++gp)
                    s += p->xfer[gp * p->G + g] * p->sigs[(long)gp * nc + c] * phi[((long)gp * nc + c) * 8 + n];
                S[((long)g * nc + c) * 8 + n] = s / (4.0 * PI);
            }
}

/* ------------------------------------------------------------------------ */
/* Source iteration (Sec. 2, after Eq. (7) and after Eq. (14)): build the   */
/* source from phi, sweep, update phi, until the change is below tol.        */
/* Change measures: max_{g,c,n} |phi_new - phi_old| / max |phi_new|, and the */
/* mean form of Eq. (21) over cells (cell-averaged phi, all groups).         */
/* The stop test uses the max form.  phi holds the guess and the result.     */
/* Returns 0, 1 if maxit was reached, or -1 on a solve failure.             */
/* ------------------------------------------------------------------------ */
int or_source_iterate(const or_problem *p, double tol, int maxit, double *phi, int *iters,
                      double *chg_max, double *chg_mean, double *tal)
{
    const long nc = ncell_of(p), n = (long)p->G * nc * 8;
    double *S = (double *)malloc(sizeof(double) * n);
    double *pn = (double *)malloc(sizeof(double) * n);
    int rc = 1;
    *iters = 0;
    for (int it = 0; it < maxit; ++it) {
        or_source(p, phi, S);
        double t[4] = {0, 0, 0, 0};
        if (or_sweep(p, S, pn, 0, p->G, 0, p->ndir, t) != 0) { rc = -1; break; }
        double dmax = 0.0, pmax = 0.0, mean = 0.0;
        for (long i = 0; i < n; ++i) {
            double dd = fabs(pn[i] - phi[i]);
            if (dd > dmax) dmax = dd;
            if (fabs(pn[i]) > pmax) pmax = fabs(pn[i]);
        }
        long cnt = 0;
        for (int g = 0; g < p->G; ++g)
            for (long c = 0; c < nc; ++c) {
                double a = 0.0, b = 0.0;
                for (int k = 0; k < 8; ++k) {
                    a += pn[((long)g * nc + c) * 8 + k];
                    b += phi[((long)g * nc + c) * 8 + k];
                }
                if (a != 0.0) { mean += fabs(a - b) / fabs(a); ++cnt; }
            }
        memcpy(phi, pn, sizeof(double) * n);
        *iters = it + 1;
        *chg_max = pmax > 0.0 ? dmax / pmax : 0.0;
        *chg_mean = cnt ? mean / cnt : 0.0;
        if (tal) for (int m = 0; m < 4; ++m) tal[m] = t[m];
        if (*chg_max <= tol) { rc = 0; break; }
    }
    free(S);
    free(pn);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Anisotropic scattering (Eqs. (3)-(8)).  The differential scattering      */
/* cross section is expanded in Legendre polynomials up to order L,          */
/* sigma_s(mu0) = sum_n (2n+1)/(4 pi) sigma_{s,n} P_n(mu0), and by the        */
/* addition theorem the scattering source of direction Omega is              */
/* sum_{n,m} sigma_{s,n} Y_nm(Omega) phi_nm with the flux moments             */
/* phi_nm = sum_d w_d Y_nm(Omega_d) psi_d (real orthonormal harmonics).       */
/* Here the harmonics come in scaled by sqrt(4 pi), Yh = sqrt(4 pi) Y, so     */
/* that Yh_00 = 1 and moment 0 is the scalar flux: flux moments              */
/* phih_k = sum_d w_d Yh_k(Omega_d) psi_d, source moments                     */
/* Sh_k = (sum_g' xfer[g'][g] sigma_{s,n(k),g'} phih_k,g' + [k = 0] q) / 4 pi,  */
/* per-direction source S_d = sum_k Yh_k(Omega_d) Sh_k.  Moment k is (n, m)   */
/* with k = n^2 + n + m, K = (L+1)^2 moments; n(k) = floor(sqrt(k)).           */
/*   sigs_n: [L+1][G][ncell] Legendre moments sigma_{s,n} (row 0 = sigma_s)   */
/*   Yh:     [ndir][K] scaled harmonics of the problem's directions           */
/*   phi:    [G][ncell][K][8] flux moments                                    */
/* ------------------------------------------------------------------------ */
static int order_of(int k)
{
    int n = 0;
    while ((n + 1) * (n + 1) <= k) ++n;
    return n;
}

void or_source_moments(const or_problem *p, int K, const double *sigs_n, const double *phi, double *S)
{
    const long nc = ncell_of(p);
    for (int g = 0; g < p->G; ++g)
        for (long c = 0; c < nc; ++c)
            for (int k = 0; k < K; ++k) {
                const int n = order_of(k);
                for (int q = 0; q < 8; ++q) {
                    double s = k == 0 ? p->q[(long)g * nc + c] : 0.0;
                    for (int gp = 0; gp < p->G; ++gp)
                        s += p->xfer[gp * p->G + g] * sigs_n[((long)n * p->G + gp) * nc + c] *
                             phi[(((long)gp * nc + c) * K + k) * 8 + q];
                    S[(((long)g * nc + c) * K + k) * 8 + q] = s / (4.0 * PI);
                }
            }
}

/* One sweep of every direction of groups [g0, g1) from the source moments S     */
/* [G][ncell][K][8]; flux moments out [G][ncell][K][8] (zero outside the        */
/* groups); tal[4] as or_sweep.                                                 */
int or_sweep_moments(const or_problem *p, int K, const double *Yh, const double *S, double *phi, int g0, int g1,
                     double *tal)
{
    or_elem e;
    or_element(p->dx, p->dy, p->dz, e.M, e.L, e.G, e.F);
    const long nc = ncell_of(p);
    int bad = 0;
    double gt[64][4];
    memset(gt, 0, sizeof(gt));
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int g = g0; g < g1; ++g) {
        double *psi = (double *)malloc(sizeof(double) * 8 * nc);
        double *Sd = (double *)malloc(sizeof(double) * 8 * nc);
        double *ph = phi + (long)g * nc * K * 8;
        const double *Sg = S + (long)g * nc * K * 8;
        for (long i = 0; i < nc * K * 8; ++i) ph[i] = 0.0;
        for (int d = 0; d < p->ndir; ++d) {
            const double *y = Yh + (long)d * K;
            for (long c = 0; c < nc; ++c)
                for (int q = 0; q < 8; ++q) {
                    double s = 0.0;
                    for (int k = 0; k < K; ++k) s += y[k] * Sg[(c * K + k) * 8 + q];
                    Sd[c * 8 + q] = s;
                }
            double t[4] = {0, 0, 0, 0};
            if (sweep_dir(p, &e, NULL, d, g, Sd, NULL, NULL, NULL, psi, t) != 0) bad = 1;
            for (long c = 0; c < nc; ++c)
                for (int k = 0; k < K; ++k)
                    for (int q = 0; q < 8; ++q) ph[(c * K + k) * 8 + q] += p->w[d] * y[k] * psi[c * 8 + q];
            for (int m = 0; m < 4; ++m) gt[g][m] += p->w[d] * t[m];
        }
        free(psi);
        free(Sd);
    }
    if (tal)
        for (int g = g0; g < g1; ++g)
            for (int m = 0; m < 4; ++m) tal[m] += gt[g][m];
    return bad ? -1 : 0;
}

/* Source iteration with anisotropic scattering; the change norms are those of */
/* or_source_iterate taken on moment 0 (the scalar flux).                      */
int or_source_iterate_moments(const or_problem *p, int K, const double *sigs_n, const double *Yh, double tol,
                              int maxit, double *phi, int *iters, double *chg_max, double *chg_mean, double *tal)
{
    const long nc = ncell_of(p), n = (long)p->G * nc * K * 8;
    double *S = (double *)malloc(sizeof(double) * n);
    double *pn = (double *)malloc(sizeof(double) * n);
    int rc = 1;
    *iters = 0;
    for (int it = 0; it < maxit; ++it) {
        or_source_moments(p, K, sigs_n, phi, S);
        double t[4] = {0, 0, 0, 0};
        if (or_sweep_moments(p, K, Yh, S, pn, 0, p->G, t) != 0) { rc = -1; break; }
        double dmax = 0.0, pmax = 0.0, mean = 0.0;
        long cnt = 0;
        for (int g = 0; g < p->G; ++g)
            for (long c = 0; c < nc; ++c) {
                double a = 0.0, b = 0.0;
                for (int q = 0; q < 8; ++q) {
                    const long i = (((long)g * nc + c) * K) * 8 + q;
                    const double dd = fabs(pn[i] - phi[i]);
                    if (dd > dmax) dmax = dd;
                    if (fabs(pn[i]) > pmax) pmax = fabs(pn[i]);
                    a += pn[i];
                    b += phi[i];
                }
                if (a != 0.0) { mean += fabs(a - b) / fabs(a); ++cnt; }
            }
        memcpy(phi, pn, sizeof(double) * n);
        *iters = it + 1;
        *chg_max = pmax > 0.0 ? dmax / pmax : 0.0;
        *chg_mean = cnt ? mean / cnt : 0.0;
        if (tal) for (int m = 0; m < 4; ++m) tal[m] = t[m];
        if (*chg_max <= tol) { rc = 0; break; }
    }
    free(S);
    free(pn);
    return rc;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ======================================================================== */
/* Discrete adjoint (not in the paper; the gradient of a detector response  */
/* with respect to sigma_t, sigma_s and q).  With L the upwind sweep        */
/* operator of every (direction, group), Phi psi = phi (Eq. (9)), B phi the  */
/* scattering source M (1/4pi) sum_g' xfer[g'][g] sigs_g' phi_g' and Q the   */
/* external source, the converged fluxes satisfy (L - B Phi) psi = Q and the */
/* response is R = r^T phi.  The adjoint lambda solves                       */
/*   (L - B Phi)^T lambda = Phi^T r,                                          */
/* by source iteration: lambda_dg = L_dg^{-T} (w_d x_g),                     */
/* x = r + B^T lambda, and                                                    */
/*   dR/dsigma_t[g,c] = -sum_d lambda_dgc^T M_c psi_dgc                       */
/*   dR/dsigma_s[g',c] = (1/4pi) sum_g xfer[g'][g] Lam_gc^T M_c phi_g'c       */
/*   dR/dq[g,c]        = (1/4pi) Lam_gc^T M_c 1,   Lam_g = sum_d lambda_dg.  */
/* ======================================================================== */

/* L_dg^T lam = rhs for one direction and group: the transposed block system is */
/* upper triangular in the upwind order, so cells are visited downwind first,   */
/* each solving A_c^T lam_c = rhs_c + (transposed face coupling from the        */
/* downstream neighbours).                                                      */
static int adjoint_sweep_dir(const or_problem *p, const or_elem *e, int d, int g, const double *rhs, double *lam)
{
    const double *om = p->omega + 3 * d;
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const long nc = ncell_of(p);
    int fin[3], fout[3];
    for (int ax = 0; ax < 3; ++ax) {
        fin[ax] = 2 * ax + (om[ax] >= 0.0 ? 0 : 1);
        fout[ax] = 2 * ax + (om[ax] >= 0.0 ? 1 : 0);
    }
    const double S0[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const double up0[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int kk = nz - 1; kk >= 0; --kk) {
        int k = om[2] >= 0.0 ? kk : nz - 1 - kk;
        for (int jj = ny - 1; jj >= 0; --jj) {
            int j = om[1] >= 0.0 ? jj : ny - 1 - jj;
            for (int ii = nx - 1; ii >= 0; --ii) {
                int i = om[0] >= 0.0 ? ii : nx - 1 - ii;
                long c = i + (long)nx * (j + (long)ny * k);
                double b[8];
                for (int n = 0; n < 8; ++n) b[n] = rhs[8 * c + n];
                for (int ax = 0; ax < 3; ++ax) {
                    if (om[ax] == 0.0) continue;
                    int idx[3] = {i, j, k}, n3[3] = {nx, ny, nz};
                    int di = idx[ax] + (om[ax] >= 0.0 ? 1 : -1);
                    if (di < 0 || di >= n3[ax]) continue;
                    int nb[3] = {i, j, k};
                    nb[ax] = di;
                    long cd = nb[0] + (long)nx * (nb[1] + (long)ny * nb[2]);
                    /* forward: row (cd, kr) gets |Om_a| F_fin[kr][face_node(fin,t)] * psi_c[face_node(fout,t)] */
                    for (int t = 0; t < 4; ++t) {
                        double s = 0.0;
                        for (int kr = 0; kr < 8; ++kr)
                            s += e->F[fin[ax] * 64 + kr * 8 + face_node(fin[ax], t)] * lam[8 * cd + kr];
                        b[face_node(fout[ax], t)] += fabs(om[ax]) * s;
                    }
                }
                double A[64], AT[64], bb[8], x[8];
                assemble(e, om, p->sigt[(long)g * nc + c], S0, up0, A, bb);
                for (int r = 0; r < 8; ++r)
                    for (int q = 0; q < 8; ++q) AT[r * 8 + q] = A[q * 8 + r];
                if (or_ge(8, AT, b, x) != 0) return -1;
                for (int n = 0; n < 8; ++n) lam[8 * c + n] = x[n];
            }
        }
    }
    return 0;
}

/* (M v) for the cell mass matrix */
static void mass_apply(const or_elem *e, const double *v, double *out)
{
    for (int k = 0; k < 8; ++k) {
        double s = 0.0;
        for (int j = 0; j < 8; ++j) s += e->M[k * 8 + j] * v[j];
        out[k] = s;
    }
}

/* Adjoint source iteration and gradients.  phi: converged forward flux
   [G][C][8]; resp: dR/dphi [G][C][8].  Outputs Lam [G][C][8] and the
   gradients [G][C].  Groups of each sweep run in parallel (fixed order per
   group).  Returns 0, 1 if maxit was reached, -1 on a solve failure. */
int or_adjoint(const or_problem *p, const double *phi, const double *resp, double tol, int maxit, double *Lam,
               double *gsigt, double *gsigs, double *gq, int *iters)
{
    or_elem e;
    or_element(p->dx, p->dy, p->dz, e.M, e.L, e.G, e.F);
    const long nc = ncell_of(p), n = (long)p->G * nc * 8;
    const int G = p->G;
    double *x = (double *)malloc(sizeof(double) * n);
    double *Ln = (double *)malloc(sizeof(double) * n);
    int rc = 1, bad = 0;
    for (long i = 0; i < n; ++i) Lam[i] = 0.0;
    *iters = 0;
    for (int it = 0; it < maxit; ++it) {
        /* x = r + B^T Lam: x_g'c = r_g'c + (sigs_g'c / 4pi) sum_g xfer[g'][g] M Lam_gc */
        for (int gp = 0; gp < G; ++gp)
            for (long c = 0; c < nc; ++c) {
                double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0}, ml[8];
                for (int g = 0; g < G; ++g) {
                    double f = p->xfer[gp * G + g];
                    if (f == 0.0) continue;
                    mass_apply(&e, Lam + ((long)g * nc + c) * 8, ml);
                    for (int k = 0; k < 8; ++k) acc[k] += f * ml[k];
                }
                double sc = p->sigs[(long)gp * nc + c] / (4.0 * PI);
                for (int k = 0; k < 8; ++k)
                    x[((long)gp * nc + c) * 8 + k] = resp[((long)gp * nc + c) * 8 + k] + sc * acc[k];
            }
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
        for (int g = 0; g < G; ++g) {
            double *lam = (double *)malloc(sizeof(double) * 8 * nc);
            double *rhs = (double *)malloc(sizeof(double) * 8 * nc);
            double *out = Ln + (long)g * nc * 8;
            for (long i = 0; i < 8 * nc; ++i) out[i] = 0.0;
            for (int d = 0; d < p->ndir; ++d) {
                for (long i = 0; i < 8 * nc; ++i) rhs[i] = p->w[d] * x[(long)g * nc * 8 + i];
                if (adjoint_sweep_dir(p, &e, d, g, rhs, lam) != 0) bad = 1;
                for (long i = 0; i < 8 * nc; ++i) out[i] += lam[i];
            }
            free(lam);
            free(rhs);
        }
        if (bad) { rc = -1; break; }
        double dmax = 0.0, pmax = 0.0;
        for (long i = 0; i < n; ++i) {
            double dd = fabs(Ln[i] - Lam[i]);
            if (dd > dmax) dmax = dd;
            if (fabs(Ln[i]) > pmax) pmax = fabs(Ln[i]);
        }
        memcpy(Lam, Ln, sizeof(double) * n);
        *iters = it + 1;
        if (pmax == 0.0 || dmax <= tol * pmax) { rc = 0; break; }
    }
    if (rc < 0) { free(x); free(Ln); return rc; }
    /* the adjoint source at the converged Lam */
    for (int gp = 0; gp < G; ++gp)
        for (long c = 0; c < nc; ++c) {
            double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0}, ml[8];
            for (int g = 0; g < G; ++g) {
                double f = p->xfer[gp * G + g];
                if (f == 0.0) continue;
                mass_apply(&e, Lam + ((long)g * nc + c) * 8, ml);
                for (int k = 0; k < 8; ++k) acc[k] += f * ml[k];
            }
            double sc = p->sigs[(long)gp * nc + c] / (4.0 * PI);
            for (int k = 0; k < 8; ++k)
                x[((long)gp * nc + c) * 8 + k] = resp[((long)gp * nc + c) * 8 + k] + sc * acc[k];
        }
    /* dR/dq and dR/dsigma_s from Lam */
    for (int g = 0; g < G; ++g)
        for (long c = 0; c < nc; ++c) {
            double ml[8];
            mass_apply(&e, Lam + ((long)g * nc + c) * 8, ml);
            double s = 0.0;
            for (int k = 0; k < 8; ++k) s += ml[k];
            gq[(long)g * nc + c] = s / (4.0 * PI);
        }
    for (int gp = 0; gp < G; ++gp)
        for (long c = 0; c < nc; ++c) {
            double mp[8], s = 0.0;
            mass_apply(&e, phi + ((long)gp * nc + c) * 8, mp);
            for (int g = 0; g < G; ++g) {
                double f = p->xfer[gp * G + g];
                if (f == 0.0) continue;
                const double *lg = Lam + ((long)g * nc + c) * 8;
                for (int k = 0; k < 8; ++k) s += f * lg[k] * mp[k];
            }
            gsigs[(long)gp * nc + c] = s / (4.0 * PI);
        }
    /* dR/dsigma_t: pair each direction's adjoint and forward angular flux */
    double *S = (double *)malloc(sizeof(double) * n);
    or_source(p, phi, S);
    for (long i = 0; i < (long)G * nc; ++i) gsigt[i] = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int g = 0; g < G; ++g) {
        double *lam = (double *)malloc(sizeof(double) * 8 * nc);
        double *psi = (double *)malloc(sizeof(double) * 8 * nc);
        double *rhs = (double *)malloc(sizeof(double) * 8 * nc);
        for (int d = 0; d < p->ndir; ++d) {
            for (long i = 0; i < 8 * nc; ++i) rhs[i] = p->w[d] * x[(long)g * nc * 8 + i];
            if (adjoint_sweep_dir(p, &e, d, g, rhs, lam) != 0) bad = 1;
            if (sweep_dir(p, &e, NULL, d, g, S + (long)g * nc * 8, NULL, NULL, NULL, psi, NULL) != 0) bad = 1;
            for (long c = 0; c < nc; ++c) {
                double mp[8], s = 0.0;
                mass_apply(&e, psi + 8 * c, mp);
                for (int k = 0; k < 8; ++k) s += lam[8 * c + k] * mp[k];
                gsigt[(long)g * nc + c] -= s;
            }
        }
        free(lam);
        free(psi);
        free(rhs);
    }
    free(S);
    free(x);
    free(Ln);
    return bad ? -1 : rc;
}
