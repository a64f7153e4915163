// Host-side launchers of the device kernels.  Every launcher issues work on
// `st` only and returns the launch error (cudaSuccess on success).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

// Element-operator flags for launch_stokes.
enum : int {
  OP_A = 1,    // yu += A u          (2 mu eps(u):eps(v))
  OP_BT = 2,   // yu += B^T p        (-p div v)
  OP_B = 4,    // yp  = B u          (-q div u)
};

// Stokes-family element operators on the fine or a coarse Q_k mesh.
//  u: [3][nn] velocity input (scaled per node by uscale if non-null), p: [ne][Np]
//  coef: viscosity per node (coef_nodal = 1) or per element point [ne][n^3]
//  yu: [3][nn] overwritten (zeroed first) when OP_A or OP_BT; yp: [ne][Np] overwritten when OP_B.
template <typename T>
cudaError_t launch_stokes(const Grid& g, int k, const RefTables* dtab, int ops, const T* u, const T* uscale,
                          const T* p, const T* coef, int coef_nodal, T* yu, T* yp, cudaStream_t st);

// Scalar Q_k Poisson y = L u, L = sum_d G_d^T diag(W |J| c) G_d, coefficient c per element point.
template <typename T>
cudaError_t launch_poisson(const Grid& g, int k, const RefTables* dtab, const T* u, const T* coef, T* y,
                           cudaStream_t st);

// Dense assembly (FP64) of the coarsest operators into a row-major n x n matrix indexed by
// `dof_map` (node -> dense index, -1 for eliminated nodes; vector DOFs: c * n_free_nodes + map).
cudaError_t launch_assemble_dense_A(const Grid& g, int k, const RefTables* dtab, const double* coef,
                                    int coef_nodal, const int* dof_map, int n_free_nodes, double* M, int ld,
                                    cudaStream_t st);
cudaError_t launch_assemble_dense_L_mapped(const Grid& g, int k, const RefTables* dtab, const double* coef,
                                           const int* dof_map, double* M, int ld, cudaStream_t st);
cudaError_t launch_identity_map(int n, int* m, cudaStream_t st);

// Inverse Jacobi diagonals.  diag_A: [3][nn] (0 on Dirichlet nodes); diag_L: [nn];
// diag_Kw: [ne][Np] from diag(B C^-1 B^T), cinv per node (0 on Dirichlet nodes).
template <typename T>
cudaError_t launch_dinv_A(const Grid& g, int k, const RefTables* dtab, const T* coef, int coef_nodal, T* dinv,
                          cudaStream_t st);
template <typename T>
cudaError_t launch_dinv_L(const Grid& g, int k, const RefTables* dtab, const T* coef, T* dinv, cudaStream_t st);
// per_dof = 0: cinv per node [nn], shared by the three components; 1: per DOF [3][nn].
template <typename T>
cudaError_t launch_dinv_Kw(const Grid& g, int k, const RefTables* dtab, const T* cinv, int per_dof, T* dinv,
                           cudaStream_t st);

// Lumped sqrt(mu)-weighted velocity mass M~_u(w), w = a(e) sqrt(mu), per node (FP64), and its
// inverse in T with zeros on Dirichlet nodes.
cudaError_t launch_lumped_weight(const Grid& g, int k, const RefTables* dtab, const double* mu, double a,
                                 double* out, cudaStream_t st);
// Lumped (unweighted) mass sum_{(e,q) at n} W_q |J| per node, used for the load vector.
cudaError_t launch_lumped_mass(const Grid& g, int k, const RefTables* dtab, double* out, cudaStream_t st);

// p-transfers (k >= 3) between Q1 on g1 and Q_k on the same mesh: prolong out_f (+)= P in_c,
// restrict out_c = P^T in_f (mask_dirichlet zeroes the Dirichlet vertices); ncomp stacked fields;
// dtab: the order-k tables (GLL nodes).
template <typename T>
cudaError_t launch_p_prolong(const Grid& g1, int k, const RefTables* dtab, int ncomp, const T* in_c, T* out_f, int add,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_p_restrict(const Grid& g1, int k, const RefTables* dtab, int ncomp, const T* in_f, T* out_c,
                              int mask_dirichlet, cudaStream_t st);
// p-coarsening of a per-point FP64 coefficient from Q_k ([ne][(k+1)^3], tables of order k) to Q1
// on the same mesh ([ne][8]): normalised L^2-adjoint of element-wise trilinear interpolation.
cudaError_t launch_pcoarsen_coef(const Grid& g, int k, const RefTables* dtab, const double* cf, double* cc,
                                 cudaStream_t st);
// w-BFBT weights per element point (FP64 [ne][(k+1)^3]): sqrt(mu), or with grad = 1 the
// viscosity-gradient weights (mu^2 + |grad mu|^2)^(1/4); the lumped mass M~_u(a w) per node and the
// Poisson coefficient 1 / (a(e) w) per point from them.
cudaError_t launch_weight_points(const Grid& g, int k, const RefTables* dtab, const double* mu, int grad, double* w,
                                 cudaStream_t st);
cudaError_t launch_lumped_weight_pts(const Grid& g, int k, const RefTables* dtab, const double* wp, double a,
                                     double* out, cudaStream_t st);
template <typename T>
cudaError_t launch_poisson_coef_pts(const Grid& g, int k, const double* wp, double a, T* c, cudaStream_t st);
// Coefficients: Poisson coefficient c = 1 / (a(e) sqrt(mu)) per element point; viscosity per
// element point from nodes; coarsening fine -> coarse (normalised L^2-adjoint, Sec. 6).
template <typename T>
cudaError_t launch_poisson_coef0(const Grid& g, int k, const double* mu, double a, T* c, cudaStream_t st);
template <typename T>
cudaError_t launch_nodal_to_points(const Grid& g, int k, const double* mu, T* c, cudaStream_t st);
template <typename T>
cudaError_t launch_coarsen_coef(const Grid& gf, int k, const RefTables* dtab, const T* cf, T* cc,
                                cudaStream_t st);

// Pressure transfers of the two-space Poisson V-cycle:
//   disc_to_cont: r_c = M_cd M_d^-1 r_d  ([ne][Np] -> [nn])
//   cont_to_disc: e_d = M_d^-1 M_dc e_c  ([nn] -> [ne][Np]); add = 1 accumulates into e_d.
template <typename T>
cudaError_t launch_disc_to_cont(const Grid& g, int k, const RefTables* dtab, const T* rd, T* rc, cudaStream_t st);
template <typename T>
cudaError_t launch_cont_to_disc(const Grid& g, int k, const RefTables* dtab, const T* ec, T* ed, int add,
                                cudaStream_t st);

// Nested Q_k transfers between coarse grid gc and its refinement, ncomp components of nn each.
// prolong: out_f (+)= P in_c; restrict: out_c = P^T in_f (mask_dirichlet zeroes coarse boundary).
// w1, w2: workspaces of launch_transfer_work_size(gc, k) elements per component.
size_t transfer_work_size(const Grid& gc, int k);
template <typename T>
cudaError_t launch_prolong(const Grid& gc, int k, const RefTables* dtab, int ncomp, const T* in_c, T* out_f,
                           int add, T* w1, T* w2, cudaStream_t st);
template <typename T>
cudaError_t launch_restrict(const Grid& gc, int k, const RefTables* dtab, int ncomp, const T* in_f, T* out_c,
                            int mask_dirichlet, T* w1, T* w2, cudaStream_t st);

// Multi-sinker viscosity / forcing (Sec. 2.1) at the brick's nodes, or at the given nodal
// coordinates X [3][nn] (mapped meshes); the brick's nodal coordinates; the load vector
// F = lumped_mass * f (masked).
cudaError_t launch_sinker(const Grid& g, int k, const RefTables& htab, const double* centres, int ns,
                          double omega, double delta, double dr, double beta, double* mu, double* f,
                          cudaStream_t st, const double* X = nullptr);
cudaError_t launch_node_coords(const Grid& g, int k, const RefTables& htab, double* X, cudaStream_t st);
cudaError_t launch_load_vector(const Grid& g, const double* lm, const double* f, double* F, cudaStream_t st);

// Zero the boundary-node entries of ncomp stacked nodal fields.
template <typename T>
cudaError_t launch_mask_boundary(const Grid& g, int ncomp, T* v, cudaStream_t st);

// Power-iteration start vector: counter-based SplitMix64 uniforms in [-0.5, 0.5).
template <typename T>
cudaError_t launch_splitmix_start(long long n, unsigned long long seed, T* v, cudaStream_t st);

// Inverse-viscosity lumped pressure mass (Sec. 1.3, Eq. lumping), the Schur baseline of Sec. 4:
// S[e] = T diag(1/d') T^T per element ([ne][Np][Np], FP64) from nodal mu, or with diag = 1 the
// inverse diagonal of M_p(1/mu) in the centred basis; block apply y = S r.
cudaError_t launch_mass_lumped_inv(const Grid& g, int k, const RefTables* dtab, const double* mu, int diag,
                                   double* S, cudaStream_t st);
template <typename T>
cudaError_t launch_block_apply(long long ne, int np, const T* S, const T* r, T* y, cudaStream_t st);
