/*
 * oracle.h -- declarations of the FP64 CPU oracle of the platelet
 * fluid-structure step (Wu, Xu, Kim, Alber, "Three-dimensional multiscale
 * model of deformable platelets adhesion to vessel wall in blood flow").
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, double-precision
 * restatement of the paper's equations.  It shares no code, header, table or
 * helper with the CUDA library; only tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.
 *
 * Conventions (all lattice units: h = 1, dt = 1, rho0 = 1):
 *   grid (nx, ny, nz); cell (i, j, k) has linear index (k*ny + j)*nx + i;
 *   x, y periodic; halfway walls at z = -1/2 (still) and z = nz - 1/2
 *   (moving with u_top).  Fields are structure-of-arrays:
 *   f[q*N + cell], g[d*N + cell], X[d*M + m].
 */
#ifndef PLATELET_ORACLE_H
#define PLATELET_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Host threads of the parallel loops over independent cells and nodes
 * (results do not depend on the count). */
void ora_set_threads(int n);
int ora_get_threads(void);

/* ---------------- Philox4x32-10 (Salmon et al., SC'11) ---------------- */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* 53-bit uniform in [0,1) from counter (site, step_lo, step_hi, purpose). */
double ora_uniform(uint64_t seed, uint32_t site, uint64_t step, uint32_t purpose);

/* ---------------- Lattice Boltzmann, Section 3.3 ---------------- */
typedef struct {
    int nx, ny, nz;
    double tau;        /* BGK relaxation time, Eq. 16 */
    double u_top[3];   /* velocity of the moving top wall */
    double body[3];    /* uniform body-force density added in every cell */
    int walls;         /* 0: halfway bounce-back (walls at z = -1/2, nz - 1/2);
                          1: on-site velocity walls of Eq. 23-30 (walls on the
                          node planes k = 0 and k = nz - 1) */
} ora_lb_params;

int ora_lb_q(void);
void ora_lb_lattice(int c[19 * 3], double w[19]);
/* Post-collision state of the linear shear profile between the walls:
 * u = u_top (k + 1/2)/nz (bounce-back walls) or u_top k/(nz - 1) (on-site). */
void ora_lb_init_shear(const ora_lb_params* p, double* f);
/* One step: stream (periodic x,y; halfway bounce-back at the z walls) and
 * BGK-collide with Guo forcing.  f_in/f_out are post-collision states;
 * g (3*N, may be NULL) is the spread force density; rho/v (may be NULL)
 * receive the density and the force-corrected velocity of the step. */
void ora_lb_step(const ora_lb_params* p, const double* f_in, const double* g,
                 double* f_out, double* rho, double* v);

/* ---------------- Immersed boundary, Section 3.4.2 ---------------- */
double ora_phi(double r);
void ora_ib_spread(const ora_lb_params* p, int M, const double* X, const double* F, double* g);
void ora_ib_interp(const ora_lb_params* p, int M, const double* X, const double* v, double* U);

/* ---------------- Hybrid membrane, Section 3.1 ---------------- */
typedef struct {
    double k_spring;            /* Eq. 2 */
    double k_s, k_t;            /* Eq. 4: global and local area */
    double k_v;                 /* Eq. 5 */
    double k_b;                 /* dihedral bending modulus */
    double morse_D, morse_a;    /* SCE Morse pairs */
    double rep_F0, rep_tau;     /* wall repulsion, Section 3.4.1 */
    double rep_eps_min, z_wall;
} ora_mem_params;

typedef struct ora_mesh ora_mesh;
ora_mesh* ora_mesh_create(int n_nodes, int n_tri, const int* tri, int n_pairs,
                          const int* pairs, int n_plt, const int* node_plt,
                          const unsigned char* is_membrane, const double* X0);
void ora_mesh_destroy(ora_mesh* m);
int ora_mesh_n_edges(const ora_mesh* m);
/* Per-platelet total area and enclosed volume. */
void ora_mesh_measure(const ora_mesh* m, const double* X, double* S, double* V);
/* terms[7] = spring, local area, global area, volume, bending, Morse, wall. */
void ora_mesh_energy(const ora_mesh* m, const ora_mem_params* p, const double* X, double* terms);
/* F = -grad(total energy), overwritten. */
void ora_mesh_forces(const ora_mesh* m, const ora_mem_params* p, const double* X, double* F);

/* ---------------- Adhesion (DAM), Section 3.2 ---------------- */
typedef struct {
    int lig_i0, lig_j0, lig_ni, lig_nj;   /* ligand patch on the wall plane */
    int box_nx, box_ny;                    /* periodic lengths */
    int max_per_ligand;                    /* 4 */
    double z_wall;
    double sigma, l_b, d_capture;          /* Eq. 13-14 */
    double gamma, kT;                      /* Eq. 12-13 */
    double kon0_dt, koff0_dt;
    uint64_t seed;
} ora_bond_params;

void ora_bond_forces(const ora_bond_params* p, int n_sites, const int* site_tri,
                     const double* site_w, const int* tri, int M, const int* bound,
                     const double* X, double* F);
void ora_bonds_step(const ora_bond_params* p, int n_sites, const int* site_tri,
                    const double* site_w, const int* tri, int M, const double* X,
                    int* bound, int* lig_count, uint64_t step, const int* partner, int* n_events);

/* ---------------- Platelet-platelet bridges (Section 3.2, "similarly") ---- */
typedef struct {
    double sigma, l_b, d_capture;          /* spring, rest length, capture distance */
    double gamma, kT;                      /* Eq. 12-13 */
    double kon0_dt, koff0_dt;
    int box_nx, box_ny;                    /* periodic lengths */
    uint64_t seed;
} ora_bridge_params;

double ora_pair_uniform(uint64_t seed, uint32_t i, uint32_t j, uint64_t step, uint32_t purpose);
void ora_bridge_forces(const ora_bridge_params* p, int n_sites, const int* site_tri,
                       const double* site_w, const int* tri, int M, const int* partner,
                       const double* X, double* F);
void ora_bridges_step(const ora_bridge_params* p, int n_sites, const int* site_tri,
                      const double* site_w, const int* tri, const int* site_plt, int M,
                      const double* X, const int* bound, int* partner, uint64_t step, int* n_events);

#ifdef __cplusplus
}
#endif
#endif
