/*
 * pf_oracle.h -- plain, slow, single-threaded FP64 CPU oracle of the phase-field
 * curvature energy F_eps of Song, "Generation of tubular and membranous shape
 * textures with curvature functionals" (arXiv 2103.04856).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the checker the CUDA path is compared
 * against.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant with the
 * CUDA library, and includes nothing from it.
 *
 * Field layout: u[(z*ny + y)*nx + x], periodic in all three axes, spacing h.
 * Coefficients a = (a20, a11, a02, a10, a01, a00) in the paper's order with the
 * paper's convention kappa1 >= kappa2 (Sec. 2.1, eq. F; Sec. 3.2, eq. Feps).
 */
#ifndef PF_ORACLE_H
#define PF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    double h;      /* grid spacing (Sec. 4.1, implementation details)            */
    double eps;    /* phase-transition width (eq. Meps)                          */
    double xi;     /* regularisation offset of |grad u| and of x^+ (Sec. 4.1)    */
    double a[6];   /* a20, a11, a02, a10, a01, a00 (eq. F)                       */
    int well;      /* 0: W(u)=u^2(1-u)^2, wells 0 and 1; 1: W(s)=(1-s^2)^2/4 (Sec. 2.3) */
    /* extensions of Sec. 5.2 (all zero / NULL: the plain eq. Feps) */
    double mu;            /* orientation weight: eps*mu*(theta . grad u)^2 joins the integrand */
    double theta[3];      /* orientation direction (x, y, z), used as given (Sec. 5.2 takes |theta| = 1) */
    const double* a_field;/* NULL, or spatialised coefficients a(x): a_field[k*N + i] is a_k at voxel i */
    int proj;             /* 1: M = -eps P Hess u P with P = I - n (x) n (the Hessian projected on the
                           * tangent plane, the form M takes on the tanh profile, Sec. 3.1) instead
                           * of eq. Meps; 0: eq. Meps */
} pfo_problem;

/* All functions return 0 on success, -1 on invalid arguments. */

/* E = h^3 * sum_i e_i, eq. Feps evaluated with the finite differences of Sec. 4.1. */
int pfo_energy(const pfo_problem* p, const double* u, double* E);

/* Same energy plus the exact gradient g_i = dE/du_i of the discrete sum. */
int pfo_energy_and_grad(const pfo_problem* p, const double* u, double* E, double* g);

/* Per-voxel energy density e_i (so that E = h^3 * sum e_i). */
int pfo_density(const pfo_problem* p, const double* u, double* e);

/* Gradient at n selected voxels only (flat indices idx[k]); no full-grid pass.
 * Used to check very large grids one sample at a time. */
int pfo_grad_sampled(const pfo_problem* p, const double* u, int n, const long* idx, double* g);

/* One mass-projected gradient-descent step: lambda = mean(g),
 * u_out = u_in - tau*(g - lambda).  sc (may be NULL) receives
 * {E(u_in), mean(u_in), lambda, max|g|, mean|g|}. */
int pfo_step(const pfo_problem* p, const double* u_in, double* u_out, double tau, double* sc);

/* nsteps steps in place; trace (may be NULL) receives nsteps rows of the five
 * scalars of pfo_step. */
int pfo_run(const pfo_problem* p, double* u, int nsteps, double tau, double* trace);

/* Diffuse principal curvatures kappa1 >= kappa2 (eqs. kepsa, kepsb), with the
 * exact positive part and the xi-regularised |grad u|. */
int pfo_curvatures(const pfo_problem* p, const double* u, double* k1, double* k2);

/* Viability diagnostics of Sec. 4.5 with the plain central-difference
 * gradient: out = {int |eps/2 |grad u|^2 - W(u)/eps|, int (eps/2 |grad u|^2 +
 * W(u)/eps) (the Cahn-Hilliard energy, i.e. the diffuse area), their ratio
 * (the normalised discrepancy, in [0, 1]), max u, min u}; integrals are h^3
 * times the sums over voxels. */
int pfo_diagnostics(const pfo_problem* p, const double* u, double out[5]);

/* Cells of the curvature diagram (Sec. 4.1, eq. curva_diagram): the surface
 * {u = level} triangulated by marching tetrahedra on the Freudenthal split of
 * every voxel cube (the cube at voxel (x, y, z) spans to (x+1, y+1, z+1),
 * periodically), each triangle giving one record {area, kappa1, kappa2}:
 * its area (h^2 units) and the diffuse curvatures of pfo_curvatures
 * interpolated trilinearly at its barycenter.  Records come in cube order
 * (z, y, x), then tetrahedron order, then triangle order; at most cap are
 * written, *count receives the total. */
int pfo_surface_cells(const pfo_problem* p, const double* u, double level, long cap, double* cells, long* count);

/* ---- Alg. 1 (Sec. 4.1): H^-1 flow through u = div A + m0, blur, Adam ---- */
typedef struct {
    double m0;              /* mass: the mean of u                                        */
    double lr, beta1, beta2, adam_eps;   /* Adam (Sec. 4.1: 1e-3, 0.9, 0.999, no decay)   */
    double blur_sigma;      /* Gaussian blur std in voxels (Sec. 4.1: 2); 0 = no blur      */
    int blur_radius;        /* taps on each side; the caller passes ceil(3 sigma)          */
    const double* m_field;  /* NULL, or a spatialised mass m(x) (Sec. 5.2): u = div A + m(x)  */
} pfo_hflow;

/* Discrete Gaussian of std sigma, taps -R..R, normalised to sum 1: w[0..2R]. */
void pfo_gauss_weights(double sigma, int R, double* w);

/* a <- k * a in place (periodic separable Gaussian of the flow's sigma). */
int pfo_blur(const pfo_problem* p, const pfo_hflow* f, double* a);

/* ut = k * (div A + m0) (or + m(x)); A is 3 fields A_x, A_y, A_z of N voxels each (component-major). */
int pfo_hflow_field(const pfo_problem* p, const pfo_hflow* f, const double* A, double* ut);

/* G(A) = F_eps(k * (div A + m0)) and dG/dA (3 x N). */
int pfo_hflow_grad(const pfo_problem* p, const pfo_hflow* f, const double* A, double* G, double* gA);

/* nsteps Adam steps of Alg. 1 in place on A with moments m, v (3 x N) and the
 * step counter *t (incremented per step).  trace (nsteps x 5, may be NULL):
 * {G, max|dG/dA|, mean|dG/dA|, mean(ut), t}. */
int pfo_hflow_run(const pfo_problem* p, const pfo_hflow* f, double* A, double* m, double* v, int nsteps, int* t,
                  double* trace);

/* Redundant parameters b = (h2, H0, k1, alpha, kappa1_0, beta, kappa2_0) of
 * eq. redundant expanded to the reduced coefficients a. */
void pfo_b_to_a(const double b[7], double a[6]);

#ifdef __cplusplus
}
#endif
#endif
