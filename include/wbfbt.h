/*
 * wbfbt.h -- C ABI of the GB300 w-BFBT Stokes solver.
 *
 * Discretisation (Sec. 1.2): a structured brick of nx x ny x nz affine
 * hexahedra on [0,lx] x [0,ly] x [0,lz]; continuous nodal Q_k velocity on
 * Gauss-Lobatto-Legendre (GLL) nodes and discontinuous modal P_{k-1}
 * pressure (monomials xi^a eta^b zeta^c, a+b+c <= k-1, ordered by total
 * degree then lexicographically descending), k in {2, 3, 4}; (k+1)^3-point
 * GLL collocated quadrature.
 *
 * Vector layouts (all arrays contiguous, no padding):
 *   node index      n = ix + NX*(iy + NY*iz),  NX = k*nx+1, NY = k*ny+1, NZ = k*nz+1
 *   velocity  u     component-major [3][NX*NY*NZ]  (u_x of all nodes, then u_y, u_z)
 *   pressure  p     element-major   [nx*ny*nz][Np], element e = ex + nx*(ey + ny*ez),
 *                   Np = k(k+1)(k+2)/6
 *   viscosity mu    per node        [NX*NY*NZ]
 * Dirichlet velocity DOFs (every node on the boundary, Eq. dir-bc) stay in
 * storage: operator inputs there are ignored and outputs there are zero.
 *
 * Ownership: the caller owns every input and output buffer; the context owns
 * the multigrid hierarchy and all workspaces, allocated in wbfbt_create (and
 * the geometry buffers, in the first wbfbt_set_geometry) and freed in
 * wbfbt_destroy.  No other call allocates device memory.  Work is
 * stream-ordered with the stream given to wbfbt_create: each call runs after
 * all work issued on that stream before it, on an internal stream of the
 * context, and work issued on the caller's stream after the call runs after
 * it.  "device" pointers must be valid for that order.  Calls that return
 * results to the host (wbfbt_solve) synchronise.
 *
 * Errors: every call returns an int status, 0 on success, a negative
 * WBFBT_ERR_* code otherwise (see wbfbt_status_string).  No call aborts the
 * process, and no kernel waits on a flag or spins: every device loop is
 * bounded by its problem size.
 */
#ifndef WBFBT_H
#define WBFBT_H

#ifdef __cplusplus
extern "C" {
#endif

#define WBFBT_OK               0
#define WBFBT_ERR_INVALID     -1   /* bad argument: null pointer, size, order, dtype       */
#define WBFBT_ERR_CUDA        -2   /* a CUDA runtime call failed                            */
#define WBFBT_ERR_NONFINITE   -3   /* NaN or Inf met in a residual or a Krylov coefficient  */
#define WBFBT_ERR_BREAKDOWN   -4   /* Krylov breakdown (zero or negative pivot / norm)      */
#define WBFBT_ERR_MAXIT       -5   /* iteration limit reached before the tolerance          */
#define WBFBT_ERR_SETUP       -6   /* coarse factorisation failed (matrix not SPD)          */

#define WBFBT_F64 0                /* dtype / precision codes */
#define WBFBT_F32 1
#define WBFBT_MIXED 1              /* preconditioner in FP32, Krylov and coarse solve FP64 */

typedef struct {
    int nx, ny, nz;                /* elements per direction, >= 1                         */
    double lx, ly, lz;             /* brick extents, > 0                                   */
} wbfbt_mesh;

typedef struct {
    double a_l, a_r;               /* boundary amplification of Eq. bdramp (>= 1); a_r <= 0
                                      selects max(1, (N/16) 2^(k-2)), the Table 3 setting  */
    int restart;                   /* FGMRES restart length m (default 50)                 */
    int cheb_degree;               /* Chebyshev steps per smoothing (default 3, Sec. 6)    */
    int mg_min_n;                  /* coarsen while all counts are even and min > this (4) */
    int precision;                 /* WBFBT_F64 or WBFBT_MIXED                              */
    int schur_sign;                /* -1 (default): [A B^T; 0 -S~]; +1: printed block      */
    int use_graphs;                /* 1 (default): replay the preconditioner as a CUDA graph */
    int elem_kernels;              /* k = 2 element kernels (no counterpart in the paper;
                                      the results agree to rounding):
                                      WBFBT_ELEM_AUTO (default) row-segment kernels (FP32:
                                      a thread per element, FP64: a warp per element
                                      point) on levels of >= 20000 elements, else one
                                      thread per point, and the single-kernel FP32 A apply
                                      on levels of >= 32768 elements with nx >= 32;
                                      WBFBT_ELEM_POINT / WBFBT_ELEM_ROW force the two-pass
                                      per-point or row kernels everywhere (and the three-
                                      or one-pass k = 2 restriction)                        */
    int schur;                     /* Schur-complement approximation S~ in Eq. precond-stokes:
                                      WBFBT_SCHUR_WBFBT (default) w-BFBT of Eq. wbfbt with
                                      multigrid inner solves; WBFBT_SCHUR_MASS the lumped
                                      inverse-viscosity pressure mass M~_p(1/mu) of Eq. lumping
                                      (the baseline of Sec. 4), lumped in the element basis of
                                      non-negative monomials ((1+xi)/2)^a ((1+eta)/2)^b
                                      ((1+zeta)/2)^c; WBFBT_SCHUR_MASS_DIAG the diagonal of
                                      M_p(1/mu) in the pressure basis above                 */
    int arnoldi_precision;         /* precision of the K apply inside the Arnoldi process:
                                      WBFBT_F64 (default; the exact Arnoldi relation) or, for
                                      a WBFBT_MIXED context only, WBFBT_F32 (the fused K apply
                                      on the FP32 preconditioner output); the true residual
                                      F - K x at every restart and at exit is FP64 either way,
                                      and convergence is declared on it                     */
    int weights;                   /* w-BFBT weight function w in C = M~_u(a_l w),
                                      D = M~_u(a_r w): WBFBT_WEIGHTS_SQRT_MU (default,
                                      w = sqrt(mu), Eq. wbfbt) or WBFBT_WEIGHTS_GRAD
                                      (w = (mu^2 + |grad mu|^2)^(1/4), the remark in Sec. 4;
                                      grad mu of each element's Q_k interpolant, per point);
                                      WBFBT_WEIGHTS_DIAG_A: C = D = diag(A) per DOF, the
                                      diag(A)-BFBT of Sec. 1.3 (a_l, a_r unused; the Poisson
                                      V-cycles use the coefficient 1/mu)                     */
    int kinv_cycles;               /* V-cycles per application of K~_l^-1 and K~_r^-1 inside
                                      S~^-1 (default 1, Sec. 6; 1..64): each further cycle
                                      corrects the residual, x += V(b - K_w x)             */
    int pmg;                       /* 1: p-coarsened multigrid for the viscous block A (Sec. 6,
                                      Fig. 5): Q_k on the fine mesh, then trilinear Q1 on the
                                      same mesh and on its h-coarsenings (coefficient moved to
                                      Q1 by the normalised L^2-adjoint of trilinear
                                      interpolation); 0 (default): Q_k on every level         */
    int ainv_cycles;               /* V-cycles per application of A~^-1 in Eq. precond-stokes
                                      (default 1; 1..64; Sec. 6 approximates A^-1 by V-cycles
                                      without fixing their number): each further cycle corrects
                                      the residual, x += V(b - A x)                          */
} wbfbt_opts;

#define WBFBT_SCHUR_WBFBT 0
#define WBFBT_SCHUR_MASS 1
#define WBFBT_SCHUR_MASS_DIAG 2
#define WBFBT_WEIGHTS_SQRT_MU 0
#define WBFBT_WEIGHTS_GRAD 1
#define WBFBT_WEIGHTS_DIAG_A 2

#define WBFBT_ELEM_AUTO 0
#define WBFBT_ELEM_POINT 1
#define WBFBT_ELEM_ROW 2

typedef struct wbfbt_ctx wbfbt_ctx;

/* Fill *opts with the defaults listed above. */
void wbfbt_default_opts(wbfbt_opts* opts);

/* Multi-sinker viscosity and body force of Sec. 2.1 at every velocity node.
 *   mu(x) = (DR^1/2 - DR^-1/2)(1 - chi(x)) + DR^-1/2,
 *   chi(x) = prod_i [1 - exp(-delta max(0, |x - c_i| - omega/2)^2)],
 *   f(x) = (0, 0, beta (chi(x) - 1)).
 * centres: HOST array [n_sinkers][3]; mu_out: device [nodes]; f_out: device
 * [3][nodes] (may be NULL).  FP64.  stream: a cudaStream_t (NULL = default). */
int wbfbt_sinker_setup(const wbfbt_mesh* mesh, int k, const double* centres, int n_sinkers,
                       double omega, double delta, double dr, double beta,
                       double* mu_out, double* f_out, void* stream);

/* The same fields at given node positions: X_nodes is a device array [3][nodes] (component-major,
 * the coordinates of a mapped mesh, see wbfbt_set_geometry); mesh and k give the node count.
 * Other arguments as in wbfbt_sinker_setup.  Returns WBFBT_ERR_INVALID (before any device work) if
 * X_nodes, mu_out or a non-NULL f_out is not device memory. */
int wbfbt_sinker_setup_at(const wbfbt_mesh* mesh, int k, const double* X_nodes, const double* centres,
                          int n_sinkers, double omega, double delta, double dr, double beta,
                          double* mu_out, double* f_out, void* stream);

/* The brick's node positions (GLL nodes of every element, Sec. 1.2) into the device array
 * X_out [3][nodes], component-major: the starting point of a mapped mesh.  Returns
 * WBFBT_ERR_INVALID if X_out is not device memory. */
int wbfbt_node_coords(const wbfbt_mesh* mesh, int k, double* X_out, void* stream);

/* Build a solver context: the fine operators, the sqrt(mu) lumped weights
 * C = M~_u(w_l), D = M~_u(w_r) (Eq. wbfbt, Eq. bdramp), and three multigrid
 * hierarchies (A; continuous Q_k Poisson for K_l and K_r, Sec. 6) with
 * coarsened coefficients, Jacobi diagonals, Chebyshev bounds and the FP64
 * coarsest inverses.  mu_nodes: device or host pointer [nodes], FP64, every
 * entry > 0 and finite.  opts may be NULL (defaults).  On success *out owns
 * all device memory of the solver. */
int wbfbt_create(const wbfbt_mesh* mesh, int k, const double* mu_nodes, const wbfbt_opts* opts,
                 void* stream, wbfbt_ctx** out);

/* Recompute everything that depends on the viscosity (weights, hierarchies, Jacobi
 * diagonals, Chebyshev bounds, coarsest inverses) for a new mu_nodes (device or
 * host pointer, same layout and rules as in wbfbt_create), reusing the context's
 * memory: no allocation.  This is the per-nonlinear-step setup of a Picard or
 * Newton loop, whose linearised Stokes systems share the mesh but not mu (Sec. 2). */
int wbfbt_setup(wbfbt_ctx* ctx, const double* mu_nodes);

/* Operator applies on the fine mesh, device pointers, dtype WBFBT_F64 or WBFBT_F32.
 *   apply_A  : y = A u                 (viscous stress, Sec. 1.2)          u, y [3][nodes]
 *   apply_B  : p = B u                 (divergence, b(v,q) = -int q div v) u [3][nodes], p [E][Np]
 *   apply_BT : u = B^T p               (gradient)                          p [E][Np], u [3][nodes]
 *   apply_K  : [yu; yp] = [A u + B^T p; B u]  (Eq. discrete-stokes; x = [u; p] contiguous)
 * Outputs are overwritten.  In and out must not alias. */
int wbfbt_apply_A(wbfbt_ctx* ctx, const void* u, void* y, int dtype);
int wbfbt_apply_B(wbfbt_ctx* ctx, const void* u, void* p, int dtype);
int wbfbt_apply_BT(wbfbt_ctx* ctx, const void* p, void* u, int dtype);
int wbfbt_apply_K(wbfbt_ctx* ctx, const void* x, void* y, int dtype);

/* Building blocks of the preconditioner, in the context's preconditioner precision
 * (dtype must equal WBFBT_F64 for an FP64 context, WBFBT_F32 for a mixed one):
 *   apply_Kw    : y = B C_w^-1 B^T p, which = 0 for C (w_l), 1 for D (w_r)        (Sec. 6)
 *   apply_Ainv  : y = one V-cycle for A from a zero guess                           (Sec. 6)
 *   apply_Kinv  : y = one pressure-Poisson V-cycle for K_w, which as above          (Sec. 6)
 *   apply_schur_inv : y = S~^-1 r, the w-BFBT approximation (Eq. wbfbt) with V-cycles;
 *                 r and y are projected against the constant pressure mode
 *   apply_precond   : y = [A~ B^T; 0 s S~]^-1 x  (Eq. precond-stokes), x, y = [u; p] */
int wbfbt_apply_Kw(wbfbt_ctx* ctx, int which, const void* p, void* y, int dtype);
int wbfbt_apply_Ainv(wbfbt_ctx* ctx, const void* r, void* y, int dtype);
int wbfbt_apply_Kinv(wbfbt_ctx* ctx, int which, const void* r, void* y, int dtype);
int wbfbt_apply_schur_inv(wbfbt_ctx* ctx, const void* r_p, void* y_p, int dtype);
int wbfbt_apply_precond(wbfbt_ctx* ctx, const void* x, void* y, int dtype);

/* Solve [A B^T; B 0][u; p] = [F; 0] with right-preconditioned FGMRES(m),
 * x0 = 0, until ||r|| <= rtol ||r_0|| (Euclidean, all DOFs; Sec. 1.3, Sec. 7).
 * f_nodes: body force at the nodes [3][nodes]; the load vector is
 * F_c(n) = sum_{(e,q) at n} W_q |J| f_c(x_n) (GLL quadrature), zero on the
 * Dirichlet boundary.  u [3][nodes], p [E][Np] receive the solution, p with
 * zero constant-mode mean.  f_nodes, u, p: all device or all host pointers
 * (host pointers are staged through context buffers, copies included).
 * iters / final_rel_res (may be NULL): total inner iterations and the true
 * relative residual ||F - K x|| / ||F|| in FP64 at exit.  Returns
 * WBFBT_ERR_MAXIT if maxit iterations did not reach rtol (the iterate is
 * still written). */
int wbfbt_solve(wbfbt_ctx* ctx, const double* f_nodes, double* u, double* p, double rtol, int maxit,
                int* iters, double* final_rel_res);

/* One block of the preconditioner solved on its own with FGMRES(m) to ||r|| <= rtol ||b||, x0 = 0,
 * preconditioned by that block's V-cycle (the "alone" iteration counts of Table 3, Sec. 7):
 *   WBFBT_BLOCK_A  : A x = b, velocity [3][nodes]; b's Dirichlet entries are ignored, x's are 0
 *   WBFBT_BLOCK_KL : (B C^-1 B^T) x = b, pressure [E][Np]; b and x projected against 1_psi
 *   WBFBT_BLOCK_KR : (B D^-1 B^T) x = b, as above
 * The V-cycle runs in the context's preconditioner precision (FP32 in a mixed context), the
 * Krylov vectors and the A operator in FP64, the K_w operator in the preconditioner precision.  b, x: FP64 device pointers.  iters / final_rel_res as in
 * wbfbt_solve; WBFBT_ERR_MAXIT if maxit iterations did not reach rtol (x still written).  The
 * context's Krylov workspace is reused: no allocation. */
#define WBFBT_BLOCK_A 0
#define WBFBT_BLOCK_KL 1
#define WBFBT_BLOCK_KR 2
int wbfbt_solve_block(wbfbt_ctx* ctx, int block, const double* b, double* x, double rtol, int maxit, int* iters,
                      double* final_rel_res);

/* Mapped (non-affine) hexahedral geometry.  X_nodes: the physical coordinates of every node,
 * component-major [3][nodes] (x of all nodes, then y, z), FP64, device or host pointer (copied).
 * Each element becomes the image of the reference cube under its isoparametric Q_k map
 * x(xi) = sum_a X_a l_a(xi) over its (k+1)^3 nodes, and the forms of Sec. 1.2 are integrated on
 * it: at GLL point q, du/dx = J_q^-T du/dxi with J_q = dx/dxi, weights W_q det J_q; the pressure
 * space is P_{k-1} in each element's reference coordinates.  The node numbering, the Dirichlet set
 * (the nodes on the boundary of the node grid) and the vector layouts stay those of the brick.
 * From this call on, wbfbt_apply_A / _B / _BT / _K (both dtypes), the Krylov operator and the load
 * vector of wbfbt_solve are the mapped ones; the preconditioner (every wbfbt_apply_* below
 * wbfbt_apply_K, and the block preconditioner inside wbfbt_solve) stays the brick's with the
 * context's nodal viscosity, and wbfbt_solve_block returns WBFBT_ERR_INVALID.  mu_nodes given to
 * wbfbt_create / wbfbt_setup are the viscosity at the mapped nodes.  X_nodes = NULL returns to the
 * brick.  Returns WBFBT_ERR_INVALID (and keeps the brick) if det J <= 0 or is not finite at some
 * point.  The first call allocates the geometry buffers (coordinates in FP64 and FP32, the mapped
 * lumped mass, reference tables: 44 bytes per node) in the context; later calls reuse them.
 * Synchronises. */
int wbfbt_set_geometry(wbfbt_ctx* ctx, const double* X_nodes);

/* Sizes of the context's vectors. */
int wbfbt_sizes(const wbfbt_ctx* ctx, long long* n_nodes, long long* n_elem, int* np_per_elem,
                int* n_levels);

/* Total device bytes owned by the context. */
long long wbfbt_device_bytes(const wbfbt_ctx* ctx);

/* Allocation-free form of the weighted pressure-Poisson apply, without a context:
 *   y = B C^-1 B^T p,  C = M~_u(w), w = a(e) sqrt(mu)  (a on boundary elements, 1 elsewhere).
 * The paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc -- code running under another framework's memory pool or
 * allocator hooks, real-time or embedded hosts that forbid device allocation
 * after start-up (it may synchronise the device and fragment memory), and
 * library code that may only touch caller-provided buffers.  Its temporaries
 * (C^-1 and the intermediate B^T p) live in a file-scope device array of
 * 4 * WBFBT_NOALLOC_MAX_NODES doubles (16 MiB) that every GPU loading this
 * library holds until the process exits; meshes with more than
 * WBFBT_NOALLOC_MAX_NODES velocity nodes are rejected with WBFBT_ERR_INVALID.
 * mu_nodes [nodes], p [E][Np], y [E][Np]: FP64 device pointers; y is overwritten.
 * The first call on a device, with that device current, resolves the array's
 * device address and fills the reference tables (a synchronous copy), so make
 * that first call before any stream capture.  All calls on a device share the
 * one array and leave their intermediates in it: calls that overlap on the GPU
 * (different streams, or different host threads) race and must be serialised
 * by the caller.  Returns 0 or a WBFBT_ERR_* code; never allocates. */
#define WBFBT_NOALLOC_MAX_NODES (1 << 19)
int wbfbt_apply_Kw_noalloc(const wbfbt_mesh* mesh, int k, const double* mu_nodes, double a,
                           const double* p, double* y, void* stream);

/* ---------------------------------------------------------------- learned correction
 * (not in the paper: a learned pressure-Poisson correction).  A 3-level 3-D convolutional U-Net on the
 * element grid (channels 16/32/64, 3x3x3 kernels, 2x2x2 average pooling, nearest upsampling,
 * skip concatenation [up, skip], ReLU after every convolution but the last, zero padding).
 * Tensors are voxel-major [batch][n^3][channels], voxel ex + n (ey + n ez).  Parameters are
 * FP32, flattened layer by layer (c1..c11) as W[27][cin][cout] then b[cout], tap
 * t = (dx+1) + 3 (dy+1) + 9 (dz+1):  y[v][co] = b[co] + sum_t sum_ci W[t][ci][co] x[v+d_t][ci].
 * Layers: c1 cin->16, c2 16->16, c3 16->32, c4 32->32, c5 32->64, c6 64->64, c7 96->32,
 * c8 32->32, c9 48->16, c10 16->16, c11 16->cout.  Compute in BF16 tensor-core kernels with
 * FP32 accumulation; loss = mean squared error; Adam (beta 0.9, 0.999, eps 1e-8).  n must be a
 * multiple of 4; cin, cout <= 16. */
typedef struct wbfbt_net wbfbt_net;
long long wbfbt_net_num_params(int cin, int cout);
int wbfbt_net_create(int cin, int cout, int n, int max_batch, void* stream, wbfbt_net** out);
int wbfbt_net_set_params(wbfbt_net* net, const float* theta);          /* device or host, copied */
int wbfbt_net_get_params(wbfbt_net* net, float* theta);                /* device or host          */
long long wbfbt_net_param_count(const wbfbt_net* net);
/* y = net(x): x [batch][n^3][cin], y [batch][n^3][cout], FP32 device pointers. */
int wbfbt_net_forward(wbfbt_net* net, const float* x, int batch, float* y);
/* Forward, MSE loss against target [batch][n^3][cout] and backward: *loss (host, may be NULL),
 * gradient of all parameters into grad (device or host, may be NULL); the gradient is kept
 * for wbfbt_net_adam_step. */
int wbfbt_net_loss_grad(wbfbt_net* net, const float* x, const float* target, int batch, double* loss,
                        float* grad);
int wbfbt_net_adam_step(wbfbt_net* net, float lr);
/* One convolution layer (0 = c1 ... 10 = c11) of the network in isolation, for per-layer
 * checks of the tensor-core kernels: on an n^3 grid (any n >= 1, zero padding) and `batch`
 * samples, x [batch][n^3][cin_layer] FP32 device (rounded to BF16 as the network stores its
 * activations).  If y is not NULL: y [batch][n^3][cout_layer] = bias + sum_t sum_ci W x, with
 * the layer's ReLU (c1..c10), in FP32 before the network's BF16 storage rounding.  If g and dW
 * are not NULL: g [batch][n^3][cout_layer] FP32 (rounded to BF16) and dW [27][cin][cout] the
 * weight gradient sum_{b,v} x[b][v + d_t][ci] g[b][v][co] accumulated in FP32.  The kernels are
 * the ones forward and backward use.  Allocates its BF16 temporaries and synchronises. */
int wbfbt_net_conv_layer(wbfbt_net* net, int layer, int n, int batch, const float* x, float* y, const float* g,
                         float* dW);
/* Checkpoint: parameters and Adam state, binary file with a header. */
int wbfbt_net_save(wbfbt_net* net, const char* path);
int wbfbt_net_load(wbfbt_net* net, const char* path);
void wbfbt_net_destroy(wbfbt_net* net);

/* Use `net` (or NULL to detach) for the pressure-Poisson inverses inside S~^-1: bit 1 of
 * `which_mask` for K_r = B D^-1 B^T, bit 0 for K_l = B C^-1 B^T.  Each application builds the
 * features x[e] = (mean log10 mu over the element's nodes / 4, q_e / s), q = diag(K_w)^-1/2 r,
 * s = rms(q), runs the net, forms z = s diag(K_w)^-1/2 y, and keeps z only if
 * ||r - K_w z|| < accept_ratio ||r|| (0 < accept_ratio <= 1; 1 keeps every step that reduces
 * the residual); otherwise it runs the V-cycle (the fallback).  The net's grid must be
 * the element grid (nx = ny = nz = n) and cin = 1 + Np, cout = Np.  While a net is attached
 * the preconditioner is not replayed as a graph (the acceptance test is a host decision). */
int wbfbt_attach_net(wbfbt_ctx* ctx, wbfbt_net* net, int which_mask, double accept_ratio);
/* A training pair from the solver itself: for a pressure residual r [E][Np] (FP64 device,
 * mean-free), x_out [E][1+Np] are the features above and y_out [E][Np] the V-cycle
 * correction z = K~_w^-1 r in the net's output units (y = z / (s diag(K_w)^-1/2)). */
int wbfbt_learned_sample(wbfbt_ctx* ctx, int which, const double* r, float* x_out, float* y_out);
/* Learned applications kept / replaced by the V-cycle since the context was created. */
int wbfbt_learned_stats(const wbfbt_ctx* ctx, long long* accepted, long long* rejected);
/* Load a checkpoint (wbfbt_net_save or wbfbt_train_learned) into a network owned by the context
 * (released by wbfbt_destroy or by a later call) and attach it for K_r = B D^-1 B^T with
 * accept_ratio 1, as wbfbt_attach_net does.  The element grid must be a cube whose edge count
 * is a multiple of 4.  Errors: WBFBT_ERR_INVALID (arguments, grid, checkpoint format). */
int wbfbt_load_learned(wbfbt_ctx* ctx, const char* path);
/* Train the learned correction on pairs the solver generates and write the checkpoint to
 * out_path.  cfg_json (may be NULL) is a flat JSON object with any of "fields" (viscosity
 * fields, default 100), "per_field" (residuals per field, 20), "epochs" (20), "batch" (4),
 * "lr" (1e-3, cosine decay), "seed" (1000), "init_seed" (7), "omega" (0.1), "delta" (200).
 * Field f draws 8-48 sinkers and a dynamic ratio log-uniform in [1e4, 1e8] from seed + f
 * (SplitMix64); its residuals are standard normal per coefficient with the constant mode
 * removed; the targets are the context's K_r V-cycle corrections (wbfbt_learned_sample); the
 * U-Net starts from He-normal weights and trains with Adam on shuffled mini-batches.  The call
 * allocates its pair store (fields x per_field x E x (2 Np + 1) floats) and frees it, runs
 * wbfbt_setup for every field and again with the context's own viscosity at the end, and
 * returns when the checkpoint is written.  Errors: WBFBT_ERR_INVALID (arguments, grid,
 * malformed or out-of-range configuration), WBFBT_ERR_CUDA, or the status of a failing step. */
int wbfbt_train_learned(wbfbt_ctx* ctx, const char* cfg_json, const char* out_path);

/* Number of CUDA kernels this library has launched in the process so far (all contexts). */
long long wbfbt_launch_count(void);

void wbfbt_destroy(wbfbt_ctx* ctx);
const char* wbfbt_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* WBFBT_H */
