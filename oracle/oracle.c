/*
 * oracle.c -- FP64 CPU oracle of the platelet fluid-structure step.
 *
 * TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU
 * baseline leg).  It restates, in plain loops and double precision, what
 * Wu, Xu, Kim and Alber's multiscale platelet model computes per time step:
 *   Section 3.1  hybrid membrane (Eq. 2-5, 11; bending per Eq. 6 read as a
 *                discrete dihedral Helfrich energy; SCE Morse pairs),
 *   Section 3.2  stochastic GPIb-alpha / vWF-A1 bonds (Eq. 12-14),
 *   Section 3.3  D3Q19 BGK lattice Boltzmann with Guo forcing (Eq. 16-21),
 *   Section 3.4  wall repulsion (3.4.1) and immersed-boundary coupling
 *                (3.4.2, Eq. 33-36).
 * Readings of garbled or silent passages are listed in the design notes of
 * the repository; each is marked "reading:" where it is used below.
 * No blocking, fusion or reordering beyond the equations is done here.
 * The loops over independent cells (lattice step, initial state) and nodes
 * (interpolation) may run on several host threads (OpenMP, ora_set_threads):
 * each iteration writes only its own outputs, so the results do not depend
 * on the thread count.
 */
#include "oracle.h"

#include <omp.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Host threads used by the parallel loops (at least 1). */
void ora_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int ora_get_threads(void) { return omp_get_max_threads(); }

/* ======================================================================
 * Philox4x32-10 counter-based generator, written from its published
 * definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
 * multipliers 0xD2511F53 / 0xCD9E8D57, the key bumped by the Weyl constants
 * 0x9E3779B9 / 0xBB67AE85 between rounds.
 * ==================================================================== */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k[0];
        uint32_t n2 = hi0 ^ c[3] ^ k[1];
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

/* Uniform draw for one (site, step, purpose): counter (site, step low word,
 * step high word, purpose), key = seed; 53 bits from the first two output
 * words (32 high bits from word 0, 21 from the top of word 1). */
double ora_uniform(uint64_t seed, uint32_t site, uint64_t step, uint32_t purpose)
{
    uint32_t ctr[4] = {site, (uint32_t)step, (uint32_t)(step >> 32), purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    ora_philox4x32_10(ctr, key, r);
    uint64_t bits = ((uint64_t)r[0] << 21) | (uint64_t)(r[1] >> 11);
    return (double)bits * (1.0 / 9007199254740992.0); /* 2^-53 */
}

/* ======================================================================
 * D3Q19 lattice, Section 3.3.  Directions in the paper's numbering (0-based
 * here), which Eq. 23-30 fix: 1..6 axes, 7..18 face diagonals, 19 rest.
 * Weights of Eq. 21.
 * ==================================================================== */
static const int C[19][3] = {
    {+1, 0, 0},  {-1, 0, 0},  {0, +1, 0},  {0, -1, 0},  {0, 0, +1},
    {0, 0, -1},  {+1, +1, 0}, {+1, -1, 0}, {+1, 0, +1}, {+1, 0, -1},
    {-1, +1, 0}, {-1, -1, 0}, {-1, 0, +1}, {-1, 0, -1}, {0, +1, +1},
    {0, +1, -1}, {0, -1, +1}, {0, -1, -1}, {0, 0, 0}};
static const double W[19] = {
    2.0 / 36, 2.0 / 36, 2.0 / 36, 2.0 / 36, 2.0 / 36, 2.0 / 36, 1.0 / 36,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 12.0 / 36};
static const double CS2 = 1.0 / 3.0; /* c_s^2 = 1/3 in lattice units */

int ora_lb_q(void) { return 19; }

void ora_lb_lattice(int c[19 * 3], double w[19])
{
    for (int q = 0; q < 19; ++q) {
        for (int d = 0; d < 3; ++d) c[3 * q + d] = C[q][d];
        w[q] = W[q];
    }
}

static int opposite(int q)
{
    for (int r = 0; r < 19; ++r)
        if (C[r][0] == -C[q][0] && C[r][1] == -C[q][1] && C[r][2] == -C[q][2]) return r;
    return -1;
}

static long cell_index(const ora_lb_params* p, int i, int j, int k)
{
    return ((long)k * p->ny + j) * p->nx + i;
}

/* Eq. 20: second-order equilibrium at density rho and velocity v. */
static double f_equilibrium(int q, double rho, const double v[3])
{
    double cv = C[q][0] * v[0] + C[q][1] * v[1] + C[q][2] * v[2];
    double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    return W[q] * rho * (1.0 + cv / CS2 + cv * cv / (2.0 * CS2 * CS2) - vv / (2.0 * CS2));
}

/* Eq. 19 forcing term (Guo).  Reading: the tensor is (c c^T - c_s^2 I), the
 * sign Guo et al. use (the printed "+" would create mass), and the velocity
 * in it is the force-corrected v, as in Guo et al. */
static double guo_source(int q, double tau, const double v[3], const double F[3])
{
    double Fc = F[0] * C[q][0] + F[1] * C[q][1] + F[2] * C[q][2];
    double contraction = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double vF = v[a] * F[b] + F[a] * v[b];
            double Q = (double)C[q][a] * C[q][b] - (a == b ? CS2 : 0.0);
            contraction += vF * Q;
        }
    return W[q] * (1.0 - 1.0 / (2.0 * tau)) * (Fc / CS2 + contraction / (2.0 * CS2 * CS2));
}

/* Initial post-collision state of the shear profile u(k) = u_top (k+1/2)/nz:
 * f* = f_eq(1, u) + (1 - 1/tau) f_neq with the Chapman-Enskog first-order
 * part f_neq = -tau w rho (c_a c_b - c_s^2 delta_ab) d_a u_b / c_s^2.
 * Reading: runs start from the developed profile (the viscous time of the
 * channels is far longer than the windows simulated). */
void ora_lb_init_shear(const ora_lb_params* p, double* f)
{
    long N = (long)p->nx * p->ny * p->nz;
    /* the walls sit half a link outside the end layers (bounce-back) or on
       them (on-site) */
    double H = p->walls ? (double)(p->nz - 1) : (double)p->nz;
    double z0 = p->walls ? 0.0 : 0.5;
    double dudz[3] = {p->u_top[0] / H, p->u_top[1] / H, 0.0};
#pragma omp parallel for schedule(static)
    for (int k = 0; k < p->nz; ++k)
        for (int j = 0; j < p->ny; ++j)
            for (int i = 0; i < p->nx; ++i) {
                long cell = cell_index(p, i, j, k);
                double u[3] = {dudz[0] * (k + z0), dudz[1] * (k + z0), 0.0};
                for (int q = 0; q < 19; ++q) {
                    double Qgrad = 0.0; /* Q_ab d_a u_b with only d_z u_x, d_z u_y */
                    for (int b = 0; b < 2; ++b) Qgrad += (double)C[q][2] * C[q][b] * dudz[b];
                    double fneq = -p->tau * W[q] * 1.0 * Qgrad / CS2;
                    f[q * N + cell] = f_equilibrium(q, 1.0, u) + (1.0 - 1.0 / p->tau) * fneq;
                }
            }
}

/* Index of the population with velocity (cx, cy, cz). */
static int dir_index(int cx, int cy, int cz)
{
    for (int q = 0; q < 19; ++q)
        if (C[q][0] == cx && C[q][1] == cy && C[q][2] == cz) return q;
    return -1;
}

/* On-site velocity wall of Hecht and Harting (Eq. 23-30) on a node plane
 * with wall velocity vw: the populations entering the fluid (c_z = +1 at the
 * bottom, c_z = -1 at the top) are unknown after streaming and are set from
 * the known ones.  The bottom follows Eq. 23-30 as printed (paper numbering
 * f1..f19 = q 0..18 here); the top is their mirror image z -> -z (reading:
 * the paper prints the bottom case only).  With s = +1 (bottom) or -1 (top):
 *   rho = [sum_{c_z = 0} f + 2 sum_{c_z = -s} f] / (1 - s vz)        (Eq. 23)
 *   N_x = 1/2 sum_{c_z = 0} c_x f - rho vx / 3,  N_y likewise      (Eq. 29-30)
 *   f_q = f_opp(q) + (rho/3) c_q.v                 for c_q = (0, 0, s) (Eq. 24)
 *   f_q = f_opp(q) + (rho/6) c_q.v - c_qx N_x - c_qy N_y  for the
 *         diagonals with c_qz = s                               (Eq. 25-28) */
static void onsite_wall(double* f, int s, const double* vw)
{
    double sum0 = 0.0, sum_out = 0.0, jx = 0.0, jy = 0.0;
    for (int q = 0; q < 19; ++q) {
        if (C[q][2] == 0) {
            sum0 += f[q];
            jx += C[q][0] * f[q];
            jy += C[q][1] * f[q];
        } else if (C[q][2] == -s) {
            sum_out += f[q];
        }
    }
    double rho = (sum0 + 2.0 * sum_out) / (1.0 - s * vw[2]);
    double Nx = 0.5 * jx - rho * vw[0] / 3.0;
    double Ny = 0.5 * jy - rho * vw[1] / 3.0;
    for (int q = 0; q < 19; ++q) {
        if (C[q][2] != s) continue;
        int o = dir_index(-C[q][0], -C[q][1], -C[q][2]);
        double cv = C[q][0] * vw[0] + C[q][1] * vw[1] + C[q][2] * vw[2];
        if (C[q][0] == 0 && C[q][1] == 0)
            f[q] = f[o] + rho * cv / 3.0;
        else
            f[q] = f[o] + rho * cv / 6.0 - C[q][0] * Nx - C[q][1] * Ny;
    }
}

/* One lattice Boltzmann step (Eq. 16-20).  The state between steps is the
 * post-collision distribution; a step streams it (each population moves one
 * link along c_q; periodic in x and y) and then collides with BGK plus the
 * Guo source.  Walls (p->walls = 0, reading): halfway bounce-back (a
 * population that would enter from outside is the opposite population
 * leaving the same cell), with Ladd's moving-wall term 2 w_q rho_w (c_q .
 * u_w)/c_s^2 at the top, rho_w = rho0 = 1.  Walls (p->walls = 1): the end
 * layers are wall nodes whose entering populations come from onsite_wall;
 * reading: with a force present, the wall fixes the populations' momentum
 * rho v_w and the collision then uses v = v_w + F/(2 rho) as elsewhere. */
void ora_lb_step(const ora_lb_params* p, const double* f_in, const double* g,
                 double* f_out, double* rho_out, double* v_out)
{
    long N = (long)p->nx * p->ny * p->nz;
    const double zero[3] = {0.0, 0.0, 0.0};
#pragma omp parallel for schedule(static)
    for (int k = 0; k < p->nz; ++k)
        for (int j = 0; j < p->ny; ++j)
            for (int i = 0; i < p->nx; ++i) {
                long cell = cell_index(p, i, j, k);
                double f[19];
                for (int q = 0; q < 19; ++q) {
                    int si = i - C[q][0], sj = j - C[q][1], sk = k - C[q][2];
                    if (sk < 0 || sk >= p->nz) {
                        double cu = 0.0;
                        if (sk >= p->nz)
                            cu = C[q][0] * p->u_top[0] + C[q][1] * p->u_top[1] + C[q][2] * p->u_top[2];
                        /* on-site walls overwrite this value below */
                        f[q] = f_in[opposite(q) * N + cell] + 2.0 * W[q] * 1.0 * cu / CS2;
                    } else {
                        si = (si % p->nx + p->nx) % p->nx;
                        sj = (sj % p->ny + p->ny) % p->ny;
                        f[q] = f_in[q * N + cell_index(p, si, sj, sk)];
                    }
                }
                if (p->walls && k == 0) onsite_wall(f, +1, zero);
                if (p->walls && k == p->nz - 1) onsite_wall(f, -1, p->u_top);
                /* Eq. 17-18: density and momentum. */
                double rho = 0.0, mom[3] = {0.0, 0.0, 0.0};
                for (int q = 0; q < 19; ++q) {
                    rho += f[q];
                    for (int d = 0; d < 3; ++d) mom[d] += f[q] * C[q][d];
                }
                double F[3], v[3];
                for (int d = 0; d < 3; ++d) {
                    F[d] = p->body[d] + (g ? g[d * N + cell] : 0.0);
                    v[d] = mom[d] / rho + F[d] / (2.0 * rho); /* v = u + F dt / (2 rho) */
                }
                for (int q = 0; q < 19; ++q) {
                    double feq = f_equilibrium(q, rho, v);
                    f_out[q * N + cell] = f[q] - (f[q] - feq) / p->tau + guo_source(q, p->tau, v, F);
                }
                if (rho_out) rho_out[cell] = rho;
                if (v_out)
                    for (int d = 0; d < 3; ++d) v_out[d * N + cell] = v[d];
            }
}

/* ======================================================================
 * Immersed boundary, Section 3.4.2.
 * ==================================================================== */

/* Eq. 36, the 4-point cosine kernel.  Reading: the garbled second branch is
 * zero for |r| > 2. */
double ora_phi(double r)
{
    double a = fabs(r);
    if (a <= 2.0) return 0.25 * (1.0 + cos(M_PI * r / 2.0));
    return 0.0;
}

/* Eq. 34-35 with h = 1: g_ijk += F_m phi(x_i - X)phi(y_j - Y)phi(z_k - Z),
 * summed over the cells in the kernel's support.  Reading: support cells
 * wrap in x and y and are dropped outside 0 <= k < nz. */
void ora_ib_spread(const ora_lb_params* p, int M, const double* X, const double* F, double* g)
{
    long N = (long)p->nx * p->ny * p->nz;
    for (int m = 0; m < M; ++m) {
        double x = X[m], y = X[M + m], z = X[2 * M + m];
        int bx = (int)floor(x) - 1, by = (int)floor(y) - 1, bz = (int)floor(z) - 1;
        for (int c = 0; c < 4; ++c)
            for (int b = 0; b < 4; ++b)
                for (int a = 0; a < 4; ++a) {
                    int ci = bx + a, cj = by + b, ck = bz + c;
                    if (ck < 0 || ck >= p->nz) continue;
                    double w = ora_phi(ci - x) * ora_phi(cj - y) * ora_phi(ck - z);
                    int wi = (ci % p->nx + p->nx) % p->nx;
                    int wj = (cj % p->ny + p->ny) % p->ny;
                    long cell = cell_index(p, wi, wj, ck);
                    for (int d = 0; d < 3; ++d) g[d * N + cell] += F[d * M + m] * w;
                }
    }
}

/* Eq. 33 with h = 1: U_m = sum over the support of v_ijk phi phi phi. */
void ora_ib_interp(const ora_lb_params* p, int M, const double* X, const double* v, double* U)
{
    long N = (long)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (int m = 0; m < M; ++m) {
        double x = X[m], y = X[M + m], z = X[2 * M + m];
        int bx = (int)floor(x) - 1, by = (int)floor(y) - 1, bz = (int)floor(z) - 1;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 4; ++c)
            for (int b = 0; b < 4; ++b)
                for (int a = 0; a < 4; ++a) {
                    int ci = bx + a, cj = by + b, ck = bz + c;
                    if (ck < 0 || ck >= p->nz) continue;
                    double w = ora_phi(ci - x) * ora_phi(cj - y) * ora_phi(ck - z);
                    int wi = (ci % p->nx + p->nx) % p->nx;
                    int wj = (cj % p->ny + p->ny) % p->ny;
                    long cell = cell_index(p, wi, wj, ck);
                    for (int d = 0; d < 3; ++d) acc[d] += v[d * N + cell] * w;
                }
        for (int d = 0; d < 3; ++d) U[d * M + m] = acc[d];
    }
}

/* ======================================================================
 * Hybrid membrane, Section 3.1.
 * ==================================================================== */
struct ora_mesh {
    int n, nt, ne, np, npl;
    int* tri;       /* 3 per triangle, outward (counter-clockwise) */
    int* tri_plt;   /* platelet of each triangle */
    int* edge;      /* 4 per edge: i, j, k, l; i->j in the triangle with k, j->i with l */
    double* L0;     /* Eq. 2 rest lengths */
    double* phi0;   /* rest dihedral (torsion) angles */
    double* S0t;    /* Eq. 4 rest triangle areas */
    double* S0p;    /* Eq. 4 rest total areas */
    double* V0p;    /* Eq. 5 rest volumes */
    int* anchor;    /* one node per platelet, the origin of its volume sum */
    int* pair;      /* Morse pairs */
    double* r0;
    int* node_plt;
    unsigned char* is_mem;
};

typedef struct {
    int lo, hi, from, wing;
} dir_edge;

static int cmp_dir_edge(const void* a, const void* b)
{
    const dir_edge* x = (const dir_edge*)a;
    const dir_edge* y = (const dir_edge*)b;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
    return x->from < y->from ? -1 : (x->from > y->from);
}

static void sub3(const double* a, const double* b, double* r)
{
    r[0] = a[0] - b[0];
    r[1] = a[1] - b[1];
    r[2] = a[2] - b[2];
}
static void cross3(const double* a, const double* b, double* r)
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }

static void get_pos(const double* X, int n, int v, double* r)
{
    r[0] = X[v];
    r[1] = X[n + v];
    r[2] = X[2 * n + v];
}
static void add_force(double* F, int n, int v, const double* f, double s)
{
    F[v] += s * f[0];
    F[n + v] += s * f[1];
    F[2 * n + v] += s * f[2];
}

/* Torsion angle of the chain r1-r2-r3-r4 and its gradient (Blondel and
 * Karplus, J. Comput. Chem. 17, 1996).  For a membrane edge i-j with wings k
 * and l the chain is k-i-j-l; the bending angle between the two triangle
 * normals differs from it by a constant, which cancels in phi - phi0. */
static double torsion(const double* r1, const double* r2, const double* r3, const double* r4,
                      double grad[4][3])
{
    double F[3], G[3], H[3], A[3], B[3], BxA[3];
    sub3(r1, r2, F);
    sub3(r2, r3, G);
    sub3(r4, r3, H);
    cross3(F, G, A);
    cross3(H, G, B);
    double A2 = dot3(A, A), B2 = dot3(B, B), gn = norm3(G);
    cross3(B, A, BxA);
    double cphi = dot3(A, B) / sqrt(A2 * B2);
    double sphi = dot3(BxA, G) / (sqrt(A2 * B2) * gn);
    if (grad) {
        double FG = dot3(F, G), HG = dot3(H, G);
        for (int d = 0; d < 3; ++d) {
            grad[0][d] = -gn / A2 * A[d];
            grad[3][d] = gn / B2 * B[d];
            grad[1][d] = gn / A2 * A[d] + FG / (A2 * gn) * A[d] - HG / (B2 * gn) * B[d];
            grad[2][d] = -gn / B2 * B[d] - FG / (A2 * gn) * A[d] + HG / (B2 * gn) * B[d];
        }
    }
    return atan2(sphi, cphi);
}

static double tri_area(const double* X, int n, const int* t)
{
    double a[3], b[3], c[3], e1[3], e2[3], nn[3];
    get_pos(X, n, t[0], a);
    get_pos(X, n, t[1], b);
    get_pos(X, n, t[2], c);
    sub3(b, a, e1);
    sub3(c, a, e2);
    cross3(e1, e2, nn);
    return 0.5 * norm3(nn);
}

/* Signed tetrahedron volume (1/6) (a-o).((b-o)x(c-o)); summed over an
 * outward closed surface it is the enclosed volume for any origin o. */
static double tri_volume(const double* X, int n, const int* t, const double* o)
{
    double a[3], b[3], c[3], bc[3];
    get_pos(X, n, t[0], a);
    get_pos(X, n, t[1], b);
    get_pos(X, n, t[2], c);
    sub3(a, o, a);
    sub3(b, o, b);
    sub3(c, o, c);
    cross3(b, c, bc);
    return dot3(a, bc) / 6.0;
}

void ora_mesh_measure(const ora_mesh* m, const double* X, double* S, double* V)
{
    for (int p = 0; p < m->npl; ++p) S[p] = V[p] = 0.0;
    for (int t = 0; t < m->nt; ++t) {
        int p = m->tri_plt[t];
        double o[3];
        get_pos(X, m->n, m->anchor[p], o);
        S[p] += tri_area(X, m->n, &m->tri[3 * t]);
        V[p] += tri_volume(X, m->n, &m->tri[3 * t], o);
    }
}

ora_mesh* ora_mesh_create(int n_nodes, int n_tri, const int* tri, int n_pairs, const int* pairs,
                          int n_plt, const int* node_plt, const unsigned char* is_membrane,
                          const double* X0)
{
    ora_mesh* m = (ora_mesh*)calloc(1, sizeof(ora_mesh));
    m->n = n_nodes;
    m->nt = n_tri;
    m->np = n_pairs;
    m->npl = n_plt;
    m->tri = (int*)malloc(sizeof(int) * 3 * (n_tri > 0 ? n_tri : 1));
    memcpy(m->tri, tri, sizeof(int) * 3 * n_tri);
    m->node_plt = (int*)malloc(sizeof(int) * n_nodes);
    memcpy(m->node_plt, node_plt, sizeof(int) * n_nodes);
    m->is_mem = (unsigned char*)malloc(n_nodes);
    memcpy(m->is_mem, is_membrane, n_nodes);
    m->tri_plt = (int*)malloc(sizeof(int) * (n_tri > 0 ? n_tri : 1));
    for (int t = 0; t < n_tri; ++t) m->tri_plt[t] = node_plt[tri[3 * t]];

    /* anchor: first membrane node (lowest index) of each platelet */
    m->anchor = (int*)malloc(sizeof(int) * (n_plt > 0 ? n_plt : 1));
    for (int p = 0; p < n_plt; ++p) m->anchor[p] = -1;
    for (int v = 0; v < n_nodes; ++v)
        if (is_membrane[v] && m->anchor[node_plt[v]] < 0) m->anchor[node_plt[v]] = v;
    for (int p = 0; p < n_plt; ++p)
        if (m->anchor[p] < 0) m->anchor[p] = 0;

    /* Edges from the triangles: every directed edge of a closed, consistently
     * oriented mesh appears once in each direction. */
    int nd = 3 * n_tri;
    dir_edge* de = (dir_edge*)malloc(sizeof(dir_edge) * (nd > 0 ? nd : 1));
    for (int t = 0; t < n_tri; ++t)
        for (int e = 0; e < 3; ++e) {
            int a = tri[3 * t + e], b = tri[3 * t + (e + 1) % 3], c = tri[3 * t + (e + 2) % 3];
            dir_edge d = {a < b ? a : b, a < b ? b : a, a, c};
            de[3 * t + e] = d;
        }
    qsort(de, nd, sizeof(dir_edge), cmp_dir_edge);
    m->edge = (int*)malloc(sizeof(int) * 4 * (nd > 0 ? nd : 1));
    int ne = 0;
    for (int s = 0; s < nd;) {
        int e = s + 1;
        while (e < nd && de[e].lo == de[s].lo && de[e].hi == de[s].hi) ++e;
        int i = de[s].from, j = (de[s].from == de[s].lo) ? de[s].hi : de[s].lo;
        int k = de[s].wing, l = -1;
        for (int r = s + 1; r < e; ++r)
            if (de[r].from == j) l = de[r].wing;
        m->edge[4 * ne + 0] = i;
        m->edge[4 * ne + 1] = j;
        m->edge[4 * ne + 2] = k;
        m->edge[4 * ne + 3] = l;
        ++ne;
        s = e;
    }
    free(de);
    m->ne = ne;

    /* Rest state from X0. */
    m->L0 = (double*)malloc(sizeof(double) * (ne > 0 ? ne : 1));
    m->phi0 = (double*)malloc(sizeof(double) * (ne > 0 ? ne : 1));
    for (int e = 0; e < ne; ++e) {
        double ri[3], rj[3], rk[3], rl[3], R[3];
        get_pos(X0, n_nodes, m->edge[4 * e + 0], ri);
        get_pos(X0, n_nodes, m->edge[4 * e + 1], rj);
        sub3(rj, ri, R);
        m->L0[e] = norm3(R);
        m->phi0[e] = 0.0;
        if (m->edge[4 * e + 3] >= 0) {
            get_pos(X0, n_nodes, m->edge[4 * e + 2], rk);
            get_pos(X0, n_nodes, m->edge[4 * e + 3], rl);
            m->phi0[e] = torsion(rk, ri, rj, rl, NULL);
        }
    }
    m->S0t = (double*)malloc(sizeof(double) * (n_tri > 0 ? n_tri : 1));
    for (int t = 0; t < n_tri; ++t) m->S0t[t] = tri_area(X0, n_nodes, &tri[3 * t]);
    m->S0p = (double*)malloc(sizeof(double) * (n_plt > 0 ? n_plt : 1));
    m->V0p = (double*)malloc(sizeof(double) * (n_plt > 0 ? n_plt : 1));
    ora_mesh_measure(m, X0, m->S0p, m->V0p);

    m->pair = (int*)malloc(sizeof(int) * 2 * (n_pairs > 0 ? n_pairs : 1));
    memcpy(m->pair, pairs, sizeof(int) * 2 * n_pairs);
    m->r0 = (double*)malloc(sizeof(double) * (n_pairs > 0 ? n_pairs : 1));
    for (int s = 0; s < n_pairs; ++s) {
        double a[3], b[3], R[3];
        get_pos(X0, n_nodes, pairs[2 * s], a);
        get_pos(X0, n_nodes, pairs[2 * s + 1], b);
        sub3(b, a, R);
        m->r0[s] = norm3(R);
    }
    return m;
}

void ora_mesh_destroy(ora_mesh* m)
{
    if (!m) return;
    free(m->tri);
    free(m->tri_plt);
    free(m->edge);
    free(m->L0);
    free(m->phi0);
    free(m->S0t);
    free(m->S0p);
    free(m->V0p);
    free(m->anchor);
    free(m->pair);
    free(m->r0);
    free(m->node_plt);
    free(m->is_mem);
    free(m);
}

int ora_mesh_n_edges(const ora_mesh* m) { return m->ne; }

/* Wall repulsion of Section 3.4.1, F = F0 tau e^{-tau eps}/(1 - e^{-tau eps}),
 * which is -dU/deps of U = -F0 ln(1 - e^{-tau eps}).  Reading: F0 carries
 * force x length; eps is clamped at eps_min (the force is held constant
 * below it and the energy continued linearly). */
static double wall_force(const ora_mem_params* p, double eps)
{
    if (eps < p->rep_eps_min) eps = p->rep_eps_min;
    double e = exp(-p->rep_tau * eps);
    return p->rep_F0 * p->rep_tau * e / (1.0 - e);
}
static double wall_energy(const ora_mem_params* p, double eps)
{
    if (eps >= p->rep_eps_min) return -p->rep_F0 * log(1.0 - exp(-p->rep_tau * eps));
    double e0 = -p->rep_F0 * log(1.0 - exp(-p->rep_tau * p->rep_eps_min));
    return e0 - wall_force(p, p->rep_eps_min) * (eps - p->rep_eps_min);
}

void ora_mesh_energy(const ora_mesh* m, const ora_mem_params* p, const double* X, double* terms)
{
    int n = m->n;
    for (int t = 0; t < 7; ++t) terms[t] = 0.0;
    /* Eq. 2: harmonic cytoskeleton springs on the mesh edges */
    for (int e = 0; e < m->ne; ++e) {
        double ri[3], rj[3], R[3];
        get_pos(X, n, m->edge[4 * e], ri);
        get_pos(X, n, m->edge[4 * e + 1], rj);
        sub3(rj, ri, R);
        double d = norm3(R) - m->L0[e];
        terms[0] += 0.5 * p->k_spring * d * d;
    }
    /* Eq. 4 (second term): local area */
    for (int t = 0; t < m->nt; ++t) {
        double d = tri_area(X, n, &m->tri[3 * t]) - m->S0t[t];
        if (p->k_t != 0.0) terms[1] += p->k_t * d * d / (2.0 * m->S0t[t]);
    }
    /* Eq. 4 (first term) and Eq. 5: global area and volume */
    double* S = (double*)malloc(sizeof(double) * m->npl);
    double* V = (double*)malloc(sizeof(double) * m->npl);
    ora_mesh_measure(m, X, S, V);
    for (int q = 0; q < m->npl; ++q) {
        double dS = S[q] - m->S0p[q], dV = V[q] - m->V0p[q];
        if (p->k_s != 0.0) terms[2] += p->k_s * dS * dS / (2.0 * m->S0p[q]);
        if (p->k_v != 0.0) terms[3] += p->k_v * dV * dV / (2.0 * m->V0p[q]);
    }
    free(S);
    free(V);
    /* Eq. 6, reading: discrete Helfrich energy k_b (1 - cos(phi - phi0)) per edge */
    for (int e = 0; e < m->ne; ++e) {
        if (m->edge[4 * e + 3] < 0) continue;
        double ri[3], rj[3], rk[3], rl[3];
        get_pos(X, n, m->edge[4 * e], ri);
        get_pos(X, n, m->edge[4 * e + 1], rj);
        get_pos(X, n, m->edge[4 * e + 2], rk);
        get_pos(X, n, m->edge[4 * e + 3], rl);
        double phi = torsion(rk, ri, rj, rl, NULL);
        terms[4] += p->k_b * (1.0 - cos(phi - m->phi0[e]));
    }
    /* SCE Morse pairs: D[(1 - e^{-a(r-r0)})^2 - 1] */
    for (int s = 0; s < m->np; ++s) {
        double a[3], b[3], R[3];
        get_pos(X, n, m->pair[2 * s], a);
        get_pos(X, n, m->pair[2 * s + 1], b);
        sub3(b, a, R);
        double x = 1.0 - exp(-p->morse_a * (norm3(R) - m->r0[s]));
        terms[5] += p->morse_D * (x * x - 1.0);
    }
    /* Section 3.4.1: wall repulsion on membrane nodes */
    for (int v = 0; v < n; ++v)
        if (m->is_mem[v]) terms[6] += wall_energy(p, X[2 * n + v] - p->z_wall);
}

/* Eq. 11 with F = -grad H (reading: the printed "+" of Eq. 11 contradicts
 * the minus sign of Eq. 3). */
void ora_mesh_forces(const ora_mesh* m, const ora_mem_params* p, const double* X, double* F)
{
    int n = m->n;
    memset(F, 0, sizeof(double) * 3 * n);
    /* Eq. 3: springs */
    for (int e = 0; e < m->ne; ++e) {
        int i = m->edge[4 * e], j = m->edge[4 * e + 1];
        double ri[3], rj[3], R[3];
        get_pos(X, n, i, ri);
        get_pos(X, n, j, rj);
        sub3(rj, ri, R);
        double r = norm3(R);
        double s = p->k_spring * (r - m->L0[e]) / r;
        add_force(F, n, i, R, s);
        add_force(F, n, j, R, -s);
    }
    /* Eq. 4-5: area and volume constraints, per triangle */
    double* S = (double*)malloc(sizeof(double) * m->npl);
    double* V = (double*)malloc(sizeof(double) * m->npl);
    ora_mesh_measure(m, X, S, V);
    for (int t = 0; t < m->nt; ++t) {
        const int* tv = &m->tri[3 * t];
        int q = m->tri_plt[t];
        double P[3][3], e1[3], e2[3], nn[3], nh[3], o[3];
        for (int a = 0; a < 3; ++a) get_pos(X, n, tv[a], P[a]);
        get_pos(X, n, m->anchor[q], o);
        sub3(P[1], P[0], e1);
        sub3(P[2], P[0], e2);
        cross3(e1, e2, nn);
        double len = norm3(nn), St = 0.5 * len;
        for (int d = 0; d < 3; ++d) nh[d] = nn[d] / len;
        /* a term whose modulus is zero contributes nothing (also for open
         * test meshes, whose rest volume can be zero) */
        double cS = 0.0, cV = 0.0;
        if (p->k_t != 0.0) cS += p->k_t * (St - m->S0t[t]) / m->S0t[t];
        if (p->k_s != 0.0) cS += p->k_s * (S[q] - m->S0p[q]) / m->S0p[q];
        if (p->k_v != 0.0) cV = p->k_v * (V[q] - m->V0p[q]) / m->V0p[q];
        for (int a = 0; a < 3; ++a) {
            /* dS_t/dP_a = (1/2) nhat x (P_{a+2} - P_{a+1}) */
            double opp[3], dS[3], pb[3], pc[3], dV[3];
            sub3(P[(a + 2) % 3], P[(a + 1) % 3], opp);
            cross3(nh, opp, dS);
            /* dV/dP_a = (1/6) (P_{a+1} - o) x (P_{a+2} - o) */
            sub3(P[(a + 1) % 3], o, pb);
            sub3(P[(a + 2) % 3], o, pc);
            cross3(pb, pc, dV);
            for (int d = 0; d < 3; ++d) {
                double f = -cS * 0.5 * dS[d] - cV * dV[d] / 6.0;
                F[d * n + tv[a]] += f;
            }
        }
    }
    free(S);
    free(V);
    /* bending (dihedral reading of Eq. 6) */
    for (int e = 0; e < m->ne; ++e) {
        int l = m->edge[4 * e + 3];
        if (l < 0) continue;
        int i = m->edge[4 * e], j = m->edge[4 * e + 1], k = m->edge[4 * e + 2];
        double ri[3], rj[3], rk[3], rl[3], gr[4][3];
        get_pos(X, n, i, ri);
        get_pos(X, n, j, rj);
        get_pos(X, n, k, rk);
        get_pos(X, n, l, rl);
        double phi = torsion(rk, ri, rj, rl, gr);
        double dE = p->k_b * sin(phi - m->phi0[e]);
        int vid[4] = {k, i, j, l};
        for (int a = 0; a < 4; ++a) add_force(F, n, vid[a], gr[a], -dE);
    }
    /* Morse pairs */
    for (int s = 0; s < m->np; ++s) {
        int i = m->pair[2 * s], j = m->pair[2 * s + 1];
        double a[3], b[3], R[3];
        get_pos(X, n, i, a);
        get_pos(X, n, j, b);
        sub3(b, a, R);
        double r = norm3(R);
        double ex = exp(-p->morse_a * (r - m->r0[s]));
        double dUdr = 2.0 * p->morse_D * p->morse_a * (1.0 - ex) * ex;
        add_force(F, n, i, R, dUdr / r);
        add_force(F, n, j, R, -dUdr / r);
    }
    /* wall repulsion, +z on membrane nodes */
    for (int v = 0; v < n; ++v)
        if (m->is_mem[v]) F[2 * n + v] += wall_force(p, X[2 * n + v] - p->z_wall);
}

/* ======================================================================
 * Stochastic adhesion (DAM), Section 3.2 and 3.4.1.
 * Ligands sit on the lattice nodes of a patch of the wall plane; ligand id
 * = (j - lig_j0) * lig_ni + (i - lig_i0).  A receptor site is a barycentric
 * point (w0, w1, 1 - w0 - w1) of a membrane triangle (reading of the
 * "randomly distributed" point locations).
 * ==================================================================== */
static void site_position(const ora_bond_params* p, const int* site_tri, const double* site_w,
                          const int* tri, int M, const double* X, int s, double* r)
{
    (void)p;
    const int* t = &tri[3 * site_tri[s]];
    double w0 = site_w[2 * s], w1 = site_w[2 * s + 1], w2 = 1.0 - w0 - w1;
    for (int d = 0; d < 3; ++d)
        r[d] = w0 * X[d * M + t[0]] + w1 * X[d * M + t[1]] + w2 * X[d * M + t[2]];
}

static double min_image(double d, int L)
{
    return d - (double)L * floor(d / (double)L + 0.5);
}

/* Vector from the ligand to the receptor (minimum image in x, y). */
/* Offset a of a ligand node from the site's node, shifted by whole box
 * lengths into the window 1 - r .. r. */
static int window_offset(int a, int box, int r)
{
    while (a > r) a -= box;
    while (a < 1 - r) a += box;
    return a;
}

static void bond_vector(const ora_bond_params* p, const double* r, int lig, double* d)
{
    int li = lig % p->lig_ni, lj = lig / p->lig_ni;
    d[0] = min_image(r[0] - (double)(p->lig_i0 + li), p->box_nx);
    d[1] = min_image(r[1] - (double)(p->lig_j0 + lj), p->box_ny);
    d[2] = r[2] - p->z_wall;
}

/* Eq. 14 (reading: a linear spring along the bond, restoring to l_b),
 * spread to the triangle's nodes with the barycentric weights. */
void ora_bond_forces(const ora_bond_params* p, int n_sites, const int* site_tri,
                     const double* site_w, const int* tri, int M, const int* bound,
                     const double* X, double* F)
{
    for (int s = 0; s < n_sites; ++s) {
        if (bound[s] < 0) continue;
        double r[3], d[3];
        site_position(p, site_tri, site_w, tri, M, X, s, r);
        bond_vector(p, r, bound[s], d);
        double xb = norm3(d);
        double c = -p->sigma * (xb - p->l_b) / xb;
        const int* t = &tri[3 * site_tri[s]];
        double w[3] = {site_w[2 * s], site_w[2 * s + 1], 1.0 - site_w[2 * s] - site_w[2 * s + 1]};
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k) F[k * M + t[a]] += w[a] * c * d[k];
    }
}

typedef struct {
    int lig, site;
} proposal;

static int cmp_proposal(const void* a, const void* b)
{
    const proposal* x = (const proposal*)a;
    const proposal* y = (const proposal*)b;
    if (x->lig != y->lig) return x->lig < y->lig ? -1 : 1;
    return x->site < y->site ? -1 : (x->site > y->site);
}

/* One Monte-Carlo adhesion update.  Reading of the event order: rupture of
 * the existing bonds first, then formation (the per-step order stated with
 * the flow chart); a site that ruptures this step stays free until the
 * next.  Rupture: P_r = 1 - exp(-k_off dt) with the Bell rate of Eq. 12,
 * F_b = sigma |x_b - l_b|.  Formation (Section 3.2: a receptor can bind a
 * ligand within the capture distance): each free site tests every ligand of
 * the patch, in ascending ligand id, that is closer than d_capture (minimum
 * image in x, y) and below capacity, with P_f = 1 - exp(-k_on dt) and k_on
 * of Eq. 13; it proposes to the lowest ligand id that succeeded.  Each
 * ligand accepts proposals in ascending site id while it has fewer than
 * max_per_ligand bonds (at most 4 receptor sites per vWF).  Draws come from
 * Philox keyed by (site, step, purpose): purpose 0 rupture; a candidate's
 * draw is named by the ligand's place in the 2r x 2r block of lattice nodes
 * around the site, r = ceil(d_capture): purpose 1 + (dj + r - 1) 2r +
 * (di + r - 1) with (di, dj) = ligand node - floor(site), wrapped into
 * 1 - r .. r (every ligand in reach lies in that block; for d_capture <= 1
 * the block is the 2x2 nodes around the site, purposes 1..4).
 * partner (may be NULL): bridge partner of each site; bridged sites are
 * not free. */
void ora_bonds_step(const ora_bond_params* p, int n_sites, const int* site_tri,
                    const double* site_w, const int* tri, int M, const double* X,
                    int* bound, int* lig_count, uint64_t step, const int* partner, int* n_events)
{
    int n_rupt = 0, n_form = 0;
    unsigned char* was_free = (unsigned char*)malloc(n_sites > 0 ? n_sites : 1);
    /* a site bridged to another platelet holds no wall bond (one bond per site) */
    for (int s = 0; s < n_sites; ++s) was_free[s] = (bound[s] < 0) && (!partner || partner[s] < 0);

    /* rupture */
    for (int s = 0; s < n_sites; ++s) {
        if (bound[s] < 0) continue;
        double r[3], d[3];
        site_position(p, site_tri, site_w, tri, M, X, s, r);
        bond_vector(p, r, bound[s], d);
        double Fb = p->sigma * fabs(norm3(d) - p->l_b);
        double koff_dt = p->koff0_dt * exp(p->gamma * Fb / p->kT);
        double Pr = -expm1(-koff_dt);
        if (ora_uniform(p->seed, (uint32_t)s, step, 0u) < Pr) {
            lig_count[bound[s]] -= 1;
            bound[s] = -1;
            ++n_rupt;
        }
    }

    /* formation proposals */
    proposal* props = (proposal*)malloc(sizeof(proposal) * (n_sites > 0 ? n_sites : 1));
    int np = 0;
    for (int s = 0; s < n_sites; ++s) {
        if (!was_free[s]) continue;
        double r[3];
        site_position(p, site_tri, site_w, tri, M, X, s, r);
        /* a bond is at least as long as the height above the wall plane:
         * no ligand is in reach above d_capture (exact for any d_capture) */
        if (!(fabs(r[2] - p->z_wall) < p->d_capture)) continue;
        double xw = r[0] - (double)p->box_nx * floor(r[0] / (double)p->box_nx);
        double yw = r[1] - (double)p->box_ny * floor(r[1] / (double)p->box_ny);
        int i0 = (int)floor(xw), j0 = (int)floor(yw);
        int rw = (int)ceil(p->d_capture);
        if (rw < 1) rw = 1;
        int best = -1;
        for (int lig = 0; lig < p->lig_ni * p->lig_nj; ++lig) {
            if (lig_count[lig] >= p->max_per_ligand) continue;
            double d[3];
            bond_vector(p, r, lig, d);
            double xb = norm3(d);
            if (!(xb < p->d_capture)) continue;
            double dev = fabs(xb - p->l_b);
            double kon_dt = p->kon0_dt * exp(p->sigma * dev * (p->gamma - 0.5 * dev) / p->kT);
            double Pf = -expm1(-kon_dt);
            int di = window_offset(p->lig_i0 + lig % p->lig_ni - i0, p->box_nx, rw);
            int dj = window_offset(p->lig_j0 + lig / p->lig_ni - j0, p->box_ny, rw);
            uint32_t purpose = (uint32_t)(1 + (dj + rw - 1) * 2 * rw + (di + rw - 1));
            double u = ora_uniform(p->seed, (uint32_t)s, step, purpose);
            if (u < Pf && best < 0) best = lig;   /* ascending id: the first success is the lowest */
        }
        if (best >= 0) {
            props[np].lig = best;
            props[np].site = s;
            ++np;
        }
    }

    /* per-ligand acceptance in ascending site id */
    qsort(props, np, sizeof(proposal), cmp_proposal);
    for (int a = 0; a < np; ++a) {
        int lig = props[a].lig;
        if (lig_count[lig] < p->max_per_ligand) {
            lig_count[lig] += 1;
            bound[props[a].site] = lig;
            ++n_form;
        }
    }
    free(props);
    free(was_free);
    n_events[0] = n_rupt;
    n_events[1] = n_form;
}

/* ======================================================================
 * Platelet-platelet bridges GPIb-alpha - vWF - GPIb-alpha (Section 3.2: the
 * paper models them "similarly" to the wall bonds and gives no equations).
 * Reading: a plasma vWF joins two receptor sites on different platelets;
 * the bridge is one linear spring between the two sites (Eq. 14 form) with
 * its own rest length, capture distance and spring constant, and the rates
 * of Eq. 12 (rupture) and Eq. 13 (formation) with those.  A site holds at
 * most one bond of either kind (steric rule 1); a bridge vWF holds exactly
 * two sites (rule 2 then holds).  Per step, after the wall update:
 *   rupture    every bridge (i < j) breaks with P_r = 1 - exp(-k_off dt),
 *              k_off of Eq. 12 with F_b = sigma |x_b - l_b|; its sites stay
 *              free until the next step;
 *   formation  every pair (i < j) of free sites on different platelets
 *              closer than d_capture succeeds with P_f = 1 - exp(-k_on dt),
 *              k_on of Eq. 13; every site picks its lowest-index successful
 *              partner, and a bridge forms where two sites picked each other.
 * Draws: Philox with counter (i, j, step low word, purpose) and key
 * (seed low word, seed high word ^ step high word) for i < j; purpose 16
 * rupture, 17 formation.  The pair vector is x_i - x_j for i < j (minimum
 * image in x, y), evaluated in that order for either site.
 * ==================================================================== */
double ora_pair_uniform(uint64_t seed, uint32_t i, uint32_t j, uint64_t step, uint32_t purpose)
{
    uint32_t ctr[4] = {i, j, (uint32_t)step, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ (uint32_t)(step >> 32)};
    uint32_t r[4];
    ora_philox4x32_10(ctr, key, r);
    uint64_t bits = ((uint64_t)r[0] << 21) | (uint64_t)(r[1] >> 11);
    return (double)bits * (1.0 / 9007199254740992.0); /* 2^-53 */
}

/* x_i - x_j, i < j, minimum image in x and y */
static void pair_vector(const ora_bridge_params* p, const double* ri, const double* rj, double* d)
{
    d[0] = min_image(ri[0] - rj[0], p->box_nx);
    d[1] = min_image(ri[1] - rj[1], p->box_ny);
    d[2] = ri[2] - rj[2];
}

void ora_bridge_forces(const ora_bridge_params* p, int n_sites, const int* site_tri,
                       const double* site_w, const int* tri, int M, const int* partner,
                       const double* X, double* F)
{
    for (int i = 0; i < n_sites; ++i) {
        int j = partner[i];
        if (j <= i) continue;
        double ri[3], rj[3], d[3];
        site_position(NULL, site_tri, site_w, tri, M, X, i, ri);
        site_position(NULL, site_tri, site_w, tri, M, X, j, rj);
        pair_vector(p, ri, rj, d);
        double xb = norm3(d);
        double c = -p->sigma * (xb - p->l_b) / xb;   /* force on site i is c d, on site j -c d */
        for (int end = 0; end < 2; ++end) {
            int s = end ? j : i;
            double sign = end ? -1.0 : 1.0;
            const int* t = &tri[3 * site_tri[s]];
            double w[3] = {site_w[2 * s], site_w[2 * s + 1], 1.0 - site_w[2 * s] - site_w[2 * s + 1]};
            for (int a = 0; a < 3; ++a)
                for (int k = 0; k < 3; ++k) F[k * M + t[a]] += sign * w[a] * c * d[k];
        }
    }
}

void ora_bridges_step(const ora_bridge_params* p, int n_sites, const int* site_tri,
                      const double* site_w, const int* tri, const int* site_plt, int M,
                      const double* X, const int* bound, int* partner, uint64_t step, int* n_events)
{
    int n_rupt = 0, n_form = 0;
    int n = n_sites > 0 ? n_sites : 1;
    double* r = (double*)malloc(sizeof(double) * 3 * n);
    unsigned char* is_free = (unsigned char*)malloc(n);
    int* choice = (int*)malloc(sizeof(int) * n);
    for (int s = 0; s < n_sites; ++s) site_position(NULL, site_tri, site_w, tri, M, X, s, &r[3 * s]);

    /* rupture; both sites of every bridge standing at the start of the step
     * stay unavailable until the next one */
    for (int s = 0; s < n_sites; ++s) is_free[s] = (partner[s] < 0);
    for (int i = 0; i < n_sites; ++i) {
        int j = partner[i];
        if (j < i) continue;
        double d[3];
        pair_vector(p, &r[3 * i], &r[3 * j], d);
        double Fb = p->sigma * fabs(norm3(d) - p->l_b);
        double koff_dt = p->koff0_dt * exp(p->gamma * Fb / p->kT);
        double Pr = -expm1(-koff_dt);
        if (ora_pair_uniform(p->seed, (uint32_t)i, (uint32_t)j, step, 16u) < Pr) {
            partner[i] = -1;
            partner[j] = -1;
            ++n_rupt;
        }
    }
    for (int s = 0; s < n_sites; ++s)
        if (bound[s] >= 0) is_free[s] = 0;

    /* formation: every site's lowest-index successful partner */
    for (int i = 0; i < n_sites; ++i) {
        choice[i] = -1;
        if (!is_free[i]) continue;
        for (int j = 0; j < n_sites; ++j) {
            if (j == i || !is_free[j] || site_plt[j] == site_plt[i]) continue;
            int a = i < j ? i : j, b = i < j ? j : i;
            double d[3];
            pair_vector(p, &r[3 * a], &r[3 * b], d);
            double xb = norm3(d);
            if (!(xb < p->d_capture)) continue;
            double dev = fabs(xb - p->l_b);
            double kon_dt = p->kon0_dt * exp(p->sigma * dev * (p->gamma - 0.5 * dev) / p->kT);
            double Pf = -expm1(-kon_dt);
            if (ora_pair_uniform(p->seed, (uint32_t)a, (uint32_t)b, step, 17u) < Pf && choice[i] < 0) choice[i] = j;
        }
    }
    for (int i = 0; i < n_sites; ++i) {
        int j = choice[i];
        if (j > i && choice[j] == i) {
            partner[i] = j;
            partner[j] = i;
            ++n_form;
        }
    }
    free(r);
    free(is_free);
    free(choice);
    n_events[0] = n_rupt;
    n_events[1] = n_form;
}
