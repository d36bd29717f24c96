/*
 * tlfe.h - C ABI of the GB300 (sm_103a) Total Lagrangian finite-element hot path.
 *
 * The operations follow "A Total Lagrangian Finite Element Framework for
 * Multibody Dynamics: Part I - Formulation" (Zhou, Arivoli, Negrut):
 *   - deformation gradient F = sum_i x_i h_i^T                 (Sec. 2.1, Eq. expression-F)
 *   - H = Hp (U Hp)^{-1}, J_p = det(U Hp), quadrature          (Sec. 6)
 *   - first Piola-Kirchhoff stress P(F, Fdot): St. Venant-Kirchhoff,
 *     compressible neo-Hookean (Mooney-Rivlin with mu01 = 0),
 *     Kelvin-Voigt damping                                      (Sec. 3.2, App. C)
 *   - internal force f_i = int P h_i dV_r                       (Sec. 4.3, Eq. internal_force_universal)
 *   - tangent K_ij = d f_i / d e_j                              (App. C, Eqs. svk_tangent, mr_tangent)
 *   - backward-Euler residual and Newton matrix                 (Sec. 7, Eq. residual; Sec. 2.2 Newton matrix)
 *
 * Conventions shared by every call
 *   - Node arrays are [n_nodes][3] row-major (x, y, z of node k at 3k..3k+2).
 *   - Displacements: the state is passed as u = x - X_ref (and its rate
 *     udot = xdot); the nodal unknowns of the paper are x = X_ref + u.
 *   - Element arrays follow the global element numbering: blocks in the order
 *     given at creation, elements of a block in their given order.
 *   - Precision: the displacement u is always double (FP64), in both
 *     precisions. A mesh created with TLFE_FP32 does its element math in FP32
 *     and takes and returns float for every other node array (udot, v, the
 *     cotangent, forces and products); TLFE_FP64 uses double throughout. FP32
 *     kernels split u into an FP32 pair (hi, lo) and form element-relative
 *     differences u_i - u_0 in FP32, so large rigid motions do not cost the
 *     strain its accuracy (F depends on u only through those differences,
 *     because sum_i h_i = 0). The Newton step state is always double.
 *   - Pointers named *_dev are CUDA device pointers, *_host host pointers.
 *     The caller owns every pointer it passes; the library never frees them and
 *     keeps none of them after the call returns (create copies what it needs).
 *   - Every call taking a stream (a cudaStream_t passed as void*, NULL = the
 *     legacy default stream) only enqueues work on it and returns; results are
 *     valid once the stream has reached that point. Calls do not synchronise
 *     unless stated.
 *   - Conditions found on the device (an inverted quadrature point, a
 *     non-finite value) are latched in the mesh's status word and returned by
 *     the next tlfe_sync (or by calls documented as synchronising).
 *   - No call aborts, traps or exits; errors are returned as tlfe_status and a
 *     thread-local message is available from tlfe_last_error().
 *   - A mesh handle may be used from one host thread at a time. Operations on
 *     one handle share its workspaces (staging buffers, the Newton state, the
 *     partial sums of TLFE_SCATTER_SORTED): issue them in one stream, or order
 *     streams with events, so that they do not run concurrently.
 */
#ifndef TLFE_H
#define TLFE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TLFE_OK = 0,
    TLFE_E_INVALID = 1,       /* bad argument, out-of-range connectivity, bad sizes */
    TLFE_E_OOM = 2,           /* device allocation failed (or host memory, while building a mesh) */
    TLFE_E_CUDA = 3,          /* a CUDA runtime call failed */
    TLFE_E_INVERTED = 4,      /* J_p <= 0 at creation, or J <= 0 (neo-Hookean) on the device */
    TLFE_E_NOT_CONVERGED = 5, /* Newton did not reach the tolerance within max_newton */
    TLFE_E_TIMEOUT = 6,       /* a bounded device-side wait ran out */
    TLFE_E_UNSUPPORTED = 7,   /* valid request the library does not implement */
    TLFE_E_NONFINITE = 8      /* NaN / Inf met on the device */
} tlfe_status;

enum { TLFE_T4 = 0, TLFE_T10 = 1, TLFE_H8 = 2, TLFE_Q27 = 3 };  /* element types (App. A; T4/H8 textbook) */
enum { TLFE_SVK = 0, TLFE_NEOHOOKE = 1, TLFE_MOONEY_RIVLIN = 2 };  /* elastic laws (Sec. 3.2, App. C) */
enum { TLFE_FP64 = 0, TLFE_FP32 = 1 };              /* element arithmetic */
/* How element contributions are summed into the node arrays:
 *   TLFE_SCATTER_ATOMIC : per tile, one atomic add per unique node and
 *                         component (fastest; summation order not fixed)
 *   TLFE_SCATTER_COLOR  : colour passes (no two elements of a pass share a
 *                         node) with plain read-add-write; deterministic
 *   TLFE_SCATTER_SORTED : every tile stores its per-node sums to a partial
 *                         buffer, then one thread per node adds that node's
 *                         partials in a fixed order; deterministic, and
 *                         close to the atomic mode in speed */
enum { TLFE_SCATTER_ATOMIC = 0, TLFE_SCATTER_COLOR = 1, TLFE_SCATTER_SORTED = 2 };
/* Where the element kernels take the reference gradients h_i from:
 *   TLFE_PATH_AUTO   : affine blocks (every T4; straight-edged T10;
 *                      parallelepiped H8 and Q27 with evenly spaced nodes)
 *                      keep J^{-1} and det J per element and
 *                      form h_i = J^{-T} dS_i/dxi(xi_q) at each point (Sec. 6,
 *                      affine case); other blocks stream the precomputed h_i
 *                      and w_q J_p of every point
 *   TLFE_PATH_SLAB   : every block streams the per-point h_i and w_q J_p
 *   TLFE_PATH_AFFINE : every block on the affine path; TLFE_E_UNSUPPORTED at
 *                      creation when a block is not affine */
enum { TLFE_PATH_AUTO = 0, TLFE_PATH_SLAB = 1, TLFE_PATH_AFFINE = 2 };
/* Order of a tile's nodes in the shared-memory node patch of the element
 * kernels (32 elements per tile; results do not depend on it):
 *   TLFE_PATCH_BANKED : nodes placed so that the 8 lanes of a quarter warp,
 *                       which read the same element-local node of their
 *                       elements in one 16-byte load, hit distinct bank
 *                       groups; nodes move only inside runs of 32 in
 *                       ascending id, so that the gather and scatter touch
 *                       the same memory sectors per warp instruction (default)
 *   TLFE_PATCH_SORTED : nodes in ascending id
 * On the T10 beam a quarter-warp patch load takes 1.04 shared-memory passes
 * banked and 1.88 sorted (tlfe_mesh_info.patch_passes). */
enum { TLFE_PATCH_BANKED = 0, TLFE_PATCH_SORTED = 1 };
/* How the element passes of one operation are launched (a property of this
 * GPU implementation; the paper has no counterpart):
 *   TLFE_LAUNCH_AUTO     : one persistent launch per operation over every pass
 *                          it covers (FP32 meshes, atomic or sorted scatter,
 *                          T4 / T10 / H8 blocks on the affine path) when there
 *                          are two or more such passes, else one launch per
 *                          pass; tlfe_autotune keeps whichever measures faster
 *   TLFE_LAUNCH_PER_PASS : one launch per pass (element block and law)
 *   TLFE_LAUNCH_FUSED    : the persistent launch wherever it covers a pass */
enum { TLFE_LAUNCH_AUTO = 0, TLFE_LAUNCH_PER_PASS = 1, TLFE_LAUNCH_FUSED = 2 };

/* One type-homogeneous element block.
 *   type  : TLFE_T4 (4 nodes), TLFE_T10 (10 nodes, App. A.1 node order),
 *           TLFE_H8 (8 nodes, tensor order i + 2j + 4k on {-1,1}^3),
 *           TLFE_Q27 (27 nodes, node i + 3j + 9k at (i-1, j-1, k-1), App. A
 *           Q27 node table)
 *   n_qp  : quadrature points per element: T4 1; T10 4 or 5; H8 8;
 *           Q27 27 (3x3x3 Gauss-Legendre)
 *   conn  : host [n_elem][nodes] 0-based global node ids (copied)
 *   body  : host [n_elem] body id in [0, n_bodies), or NULL for body 0 */
typedef struct {
    int32_t type;
    int32_t n_elem;
    int32_t n_qp;
    const int32_t *conn;
    const int32_t *body;
} tlfe_block;

/* Material of one body. model = TLFE_SVK, TLFE_NEOHOOKE or TLFE_MOONEY_RIVLIN
 * with Lame (mu, lambda). The Mooney-Rivlin law is the paper's (App. C, Eq.
 * mr_first_piola) with mu10 = mu / 2 - mu01 and bulk modulus
 * k = lambda + 2 mu / 3, so that its small-strain shear modulus
 * 2 (mu10 + mu01) is mu; the neo-Hookean law is its mu01 = 0 case (mu01 is
 * ignored for the other models). mu_v, lambda_v >= 0 are the Kelvin-Voigt
 * dissipation constants (Sec. 3.2.3; 0 = undamped). rho is the reference
 * density (used by the mass matrix and the body force). */
typedef struct {
    int32_t model;
    double mu, lambda, mu_v, lambda_v, rho;
    double mu01;
} tlfe_material;

typedef struct {
    int32_t n_nodes;
    const double *X_ref;            /* host [n_nodes][3] reference coordinates */
    int32_t n_blocks;
    const tlfe_block *blocks;       /* host [n_blocks] */
    int32_t n_bodies;
    const tlfe_material *body_mat;  /* host [n_bodies] */
    const double *elem_mu_lambda;   /* host [n_elem_total][2] per-element (mu, lambda), or NULL */
    int32_t precision;              /* TLFE_FP32 or TLFE_FP64 */
    int32_t scatter;                /* TLFE_SCATTER_ATOMIC (fast, order not fixed),
                                       TLFE_SCATTER_COLOR (deterministic colour passes) or
                                       TLFE_SCATTER_SORTED (deterministic node-ordered partial sums) */
    uint64_t color_seed;            /* priority seed of the conflict colouring */
    int32_t element_path;           /* TLFE_PATH_AUTO, TLFE_PATH_SLAB or TLFE_PATH_AFFINE */
    int32_t patch_layout;           /* TLFE_PATCH_BANKED (0) or TLFE_PATCH_SORTED */
} tlfe_mesh_desc;

typedef struct tlfe_mesh tlfe_mesh;

/* Build a mesh handle on the current CUDA device: validates connectivity and
 * sizes, uploads them, and runs the reference precompute of Section 6 on the
 * device in FP64, stored in the mesh precision: J^{-1} and det J per element
 * on the affine path, H_q = Hp(xi_q) (U Hp(xi_q))^{-1} and w_q J_p per point
 * on the slab path (see element_path). With TLFE_SCATTER_COLOR it also colours the elements
 * (Jones-Plassmann with priority splitmix64(e xor color_seed); equal to the
 * sequential greedy colouring in descending priority). Synchronises `stream`.
 * Returns TLFE_E_INVERTED if any J_p <= 0, TLFE_E_INVALID on bad input. */
tlfe_status tlfe_create_mesh(const tlfe_mesh_desc *desc, void *stream, tlfe_mesh **out);

/* Release every device array of the handle. Synchronises the device. */
tlfe_status tlfe_destroy_mesh(tlfe_mesh *mesh);

typedef struct {
    int32_t n_nodes, n_elem, n_blocks, n_colors, precision, scatter;
    int64_t n_qp;
    int64_t stream_bytes_force;   /* algorithmic bytes of one tlfe_internal_force (see design notes) */
    int64_t stream_bytes_matvec;  /* algorithmic bytes of one tlfe_tangent_matvec */
    int64_t stream_bytes_vjp;     /* algorithmic bytes of one tlfe_vjp (all outputs) */
    int64_t device_bytes;         /* device memory held by the handle */
    int32_t n_affine_blocks;      /* blocks whose kernels run on the affine path */
    int32_t n_passes;             /* tile ranges of one operation: one per elastic law of each block (per
                                     colour and law in colour mode) */
    int32_t n_fused_passes;       /* passes the fused persistent launch covers (0: no fused launch) */
    int32_t n_fused_items;        /* work items (tile runs) of the fused launch */
    int32_t launches_force;       /* kernel launches of one tlfe_internal_force in the current launch mode */
    int32_t launches_matvec;      /* kernel launches of one tlfe_tangent_matvec in the current launch mode */
    int32_t patch_layout;         /* the desc's patch_layout */
    double patch_passes;          /* shared-memory passes of one 16-byte node-patch load of a quarter warp
                                     (8 lanes reading one element-local node of their elements), averaged
                                     over the tile kernels' loads; 1 = free of bank conflicts */
    int32_t force_matvec_fused;   /* 1: tlfe_force_matvec and tlfe_step_host (with f and y requested)
                                     evaluate the force and the operator product in one pass per element
                                     block and law (FP32 meshes of T4, T10 and H8 blocks, neither
                                     operation on the persistent launch; tlfe_autotune keeps the faster
                                     of one fused pass and two passes); 0: two passes */
    int64_t stream_bytes_force_matvec;  /* algorithmic bytes of that fused pass (u, udot, v read once; f, y) */
} tlfe_mesh_info;

tlfe_status tlfe_get_mesh_info(const tlfe_mesh *mesh, tlfe_mesh_info *info);

/* Launch mode of the element passes (TLFE_LAUNCH_AUTO, TLFE_LAUNCH_PER_PASS
 * or TLFE_LAUNCH_FUSED; see their definition). Results do not depend on it
 * beyond the order of floating-point additions in the atomic scatter (the
 * sorted scatter's results are the same bit for bit). Takes effect at the
 * next call; a graph captured by tlfe_force_matvec keeps the mode it was
 * captured with until its arguments change. */
tlfe_status tlfe_set_launch_mode(tlfe_mesh *mesh, int32_t mode);

/* Colour of every element in global element order (host [n_elem]); -1 when
 * the mesh was not coloured. Synchronises. */
tlfe_status tlfe_get_colors(const tlfe_mesh *mesh, int32_t *colors_host);

/* Gather and scatter indices of the element kernels (the assembly of Sec.
 * 4.3: f_i of element e is added into the node conn[e][i]), read back from the
 * device tables the kernels use: the per-tile metadata records (unique-node
 * list, local indices, node-sorted positions), the partial-sum transpose of
 * TLFE_SCATTER_SORTED, and the connectivity of warp-per-element blocks.
 * gather_host[k] receives the node whose values the kernels load for local
 * node i of element e, scatter_host[k] the node whose entries
 * 3 node + d (d = 0, 1, 2) receive that local node's contribution, with
 * k = (offset of e's block) + (e's index in the block) * nodes + i and blocks
 * in creation order (host int32 arrays of sum over blocks of n_elem * nodes;
 * either may be NULL). A correct mesh gives conn[e][i] in both. Allocates
 * and frees scratch; synchronises the device. */
tlfe_status tlfe_get_scatter_targets(const tlfe_mesh *mesh, int32_t *gather_host, int32_t *scatter_host);

/* Wait for `stream`, read and clear the device status word.
 * n_inverted (nullable) receives the number of quadrature points that met
 * J <= 0 since the last sync. Returns TLFE_E_INVERTED / TLFE_E_NONFINITE when
 * such events were latched, else TLFE_OK. */
tlfe_status tlfe_sync(tlfe_mesh *mesh, void *stream, int64_t *n_inverted);

/* Internal force (Sec. 4.3, Eq. internal_force_universal):
 *   f_i = sum_e sum_q w_q J_p P(F_q, Fdot_q) h_{i,q},
 * F = I + sum_i u_i h_i^T, Fdot = sum_i udot_i h_i^T, P = P^e + F S^v.
 * u_dev: device double [n_nodes][3]; udot_dev: device [n_nodes][3] in the
 * mesh dtype, or NULL (no viscous stress). f_dev: device [n_nodes][3] in the
 * mesh dtype, overwritten. f_int is the restoring force (+dPi/dx). */
tlfe_status tlfe_internal_force(tlfe_mesh *mesh, const void *u_dev, const void *udot_dev,
                                void *f_dev, void *stream);

/* Same operation on HOST arrays (pageable or pinned; u double, udot and f in
 * the mesh dtype): copies u (and udot) to
 * device buffers held by the handle, evaluates, and copies f back, all on
 * `stream`. Synchronises `stream` before returning. */
tlfe_status tlfe_internal_force_host(tlfe_mesh *mesh, const void *u_host, const void *udot_host,
                                     void *f_host, void *stream);

/* Element operations of one state on HOST buffers, for callers whose data
 * live in host memory (the force of Sec. 4.3, the operator product and the
 * vector-Jacobian products below). Arrays have the layouts and dtypes of the
 * device calls: u_host double [n_nodes][3]; udot, v, cot, f, y, g_u, g_udot in
 * the mesh dtype [n_nodes][3]; g_mu_lambda double [n_elem][2]. udot may be
 * NULL. Each operation runs when its inputs and an output are given:
 *   f_host                       -> tlfe_internal_force
 *   v_host and y_host            -> tlfe_tangent_matvec (a_M, a_K, a_C)
 *   cot_host and any g_*_host    -> tlfe_vjp
 * (with f and y both requested, as one pass where tlfe_force_matvec would take
 * it, tlfe_mesh_info.force_matvec_fused)
 * Asynchronous: the call copies the inputs into one of two sets of device
 * staging buffers held by the handle (consecutive calls alternate) on a copy
 * stream of its own, runs the operations on `stream` once the inputs are in,
 * and copies each output back on a second copy stream as soon as its
 * operation has ended, so that consecutive calls overlap their transfers with
 * each other's computation. Host buffers must stay valid, and inputs
 * unchanged, until tlfe_step_host_wait returns; outputs are complete then.
 * Pinned (page-locked) host memory is needed for the copies to overlap. The
 * first call allocates the staging buffers and copy streams. */
typedef struct {
    const double *u_host;
    const void *udot_host;
    const void *v_host;
    const void *cot_host;
    double a_M, a_K, a_C;
    void *f_host;
    void *y_host;
    void *g_u_host;
    void *g_udot_host;
    double *g_mu_lambda_host;
} tlfe_host_step;

tlfe_status tlfe_step_host(tlfe_mesh *mesh, const tlfe_host_step *args, void *stream);

/* Wait until every tlfe_step_host call issued on the handle has finished,
 * its outputs written to the host buffers. */
tlfe_status tlfe_step_host_wait(tlfe_mesh *mesh);

/* Matrix-free operator product (App. C; Newton matrix of Sec. 2.2 / Sec. 7):
 *   y = a_M M v + a_K K_t(u, udot) v + a_C C(u) v
 * M: consistent mass m_ij = rho int s_i s_j dV (Sec. 4.1), K_t = d f_int / d x
 * (elastic and viscous), C = d f_int / d xdot (Kelvin-Voigt). u_dev is device
 * double [n_nodes][3]; udot_dev, v_dev and y_dev are device [n_nodes][3] in the
 * mesh dtype; udot may be NULL; y_dev is overwritten.
 * a_M != 0 needs affine elements (straight-edged tetrahedra, parallelepiped
 * bricks): TLFE_E_UNSUPPORTED otherwise. */
tlfe_status tlfe_tangent_matvec(tlfe_mesh *mesh, const void *u_dev, const void *udot_dev,
                                const void *v_dev, double a_M, double a_K, double a_C,
                                void *y_dev, void *stream);

/* Internal force and operator product of one state in one call (the force +
 * K v step of a batch of bodies: Sec. 4.3, Eq. internal_force_universal, and
 * the product above):
 *   f = f_int(u, udot),  y = a_M M v + a_K K_t(u, udot) v + a_C C(u) v
 * with the arguments and layouts of tlfe_internal_force and
 * tlfe_tangent_matvec (f and y distinct). The handle keeps a CUDA graph of
 * the call: the first call with a given set of pointers and coefficients (or
 * the first after tlfe_autotune, tlfe_set_launch_mode or the first
 * tlfe_set_elem_mu_lambda) evaluates directly and captures the same launches
 * on a stream of its own; later calls with the same arguments replay that
 * graph on `stream`. On an FP32 mesh of T4, T10 and H8 blocks the two
 * operations run as one pass per element block and law, which gathers the
 * nodal inputs and forms F, Fdot and the stress once for both outputs
 * (tlfe_mesh_info.force_matvec_fused says whether it does; tlfe_autotune keeps
 * the faster of that pass and two passes). Otherwise, in TLFE_LAUNCH_AUTO and
 * TLFE_LAUNCH_FUSED modes a mesh with a fused plan runs each operation as one
 * persistent launch. The first call with new arguments must not itself be
 * made during a stream capture. Stream-ordered; the graph is released with
 * the handle. */
tlfe_status tlfe_force_matvec(tlfe_mesh *mesh, const void *u_dev, const void *udot_dev, const void *v_dev,
                              double a_M, double a_K, double a_C, void *f_dev, void *y_dev, void *stream);

/* Diagonal of a_M M + a_K K^e + a_C C (the Jacobi preconditioner of the
 * Newton/CG step; K^e is the elastic, symmetric part of K_t).
 * d_dev: device [n_nodes][3], overwritten. */
tlfe_status tlfe_jacobi_diag(tlfe_mesh *mesh, const void *u_dev, const void *udot_dev,
                             double a_M, double a_K, double a_C, void *d_dev, void *stream);

/* External loads (Sec. 4), added into f_dev (device double [n_nodes][3],
 * caller-owned; zero it first for a fresh load vector). Both calls are
 * stream-ordered and use FP64 arithmetic with atomic accumulation.
 *
 * Pointwise forces (Eq. virtual_work_point_force_discrete): load k acts on
 * global element elem_dev[k] at parent coordinates xi_dev[k][3] with force
 * force_dev[k][3], and adds s_i(xi) force to each node i of the element.
 *
 * Surface tractions (Eq. virtual_work_traction_discrete): face k is local face
 * face_dev[k] of global element elem_dev[k], loaded by the nominal traction
 * t0_dev[k][3] (force per reference area, constant over the face); adds
 * int s_i t0 dA0 to each node of the element by boundary quadrature on the
 * reference configuration. Local faces: tetrahedra, face k is opposite corner
 * k; bricks, face 2 d + s lies at parent coordinate xi_d = -1 (s = 0) or +1
 * (s = 1). Rules: triangles 4 x 4 collapsed Gauss-Legendre, quadrilaterals
 * 3 x 3 Gauss-Legendre, dA0 = |dX/da x dX/db| da db.
 * Non-finite parent coordinates or a bad face id are counted in the status
 * word (TLFE_E_NONFINITE at the next sync) and skipped. */
tlfe_status tlfe_point_loads(tlfe_mesh *mesh, int32_t n, const int32_t *elem_dev, const double *xi_dev,
                             const double *force_dev, double *f_dev, void *stream);
tlfe_status tlfe_surface_traction(tlfe_mesh *mesh, int32_t n, const int32_t *elem_dev, const int32_t *face_dev,
                                  const double *t0_dev, double *f_dev, void *stream);

/* Bilateral constraint primitives (Sec. 3: DP1, DP2, DIST, CD), each a scalar
 * position-level condition c(q) = 0 built from point evaluations
 * r_X = sum_i s_i(xi_X) (X_i + u_i) of material points on elements:
 *   TLFE_CON_CD  : c = d . (r_Q - r_P) - f          (Eq. cd_constraint)
 *   TLFE_CON_DIST: c = 1/2 (|r_Q - r_P|^2 - f^2)    (Eq. dist_constraint)
 *   TLFE_CON_DP1 : c = (r_Q - r_P) . (r_T - r_R) - f (Eq. dp1_constraint)
 *   TLFE_CON_DP2 : the same expression with P, Q, R on one body and T on the
 *                  other (Eq. dp2_constraint)
 * Points P, Q (and R, T for DP1 / DP2): elem[k] is the global element and
 * xi[k] the parent coordinates; elem[k] < 0 makes the point a fixed ground
 * point at world coordinates xi[k]. d: CD axis; f: prescribed value f(t_{n+1})
 * (DIST: the distance). */
enum { TLFE_CON_CD = 0, TLFE_CON_DIST = 1, TLFE_CON_DP1 = 2, TLFE_CON_DP2 = 3 };
typedef struct {
    int32_t type;
    int32_t elem[4];
    double xi[4][3];
    double d[3];
    double f;
} tlfe_constraint;

/* c_dev[k] = c_k(X + u) for the n constraints cons_dev (device arrays; u_dev
 * device double [n_nodes][3], c_dev device double [n]). The first call with
 * more constraints than any call before on the handle allocates its constraint
 * scratch (kept until tlfe_destroy_mesh); later calls reuse it. All three calls
 * synchronise `stream`. Invalid elements or types: TLFE_E_INVALID. */
tlfe_status tlfe_constraint_eval(tlfe_mesh *mesh, int32_t n, const tlfe_constraint *cons_dev, const double *u_dev,
                                 double *c_dev, void *stream);
/* f_dev += C_q^T w (C_q = dc/dq at X + u, applied through the element blocks
 * of Sec. 3 without forming C_q); w_dev device double [n], f_dev device double
 * [n_nodes][3]. */
tlfe_status tlfe_constraint_jt(tlfe_mesh *mesh, int32_t n, const tlfe_constraint *cons_dev, const double *u_dev,
                               const double *w_dev, double *f_dev, void *stream);
/* out_dev[k] = (C_q v)_k; v_dev device double [n_nodes][3]. */
tlfe_status tlfe_constraint_j(tlfe_mesh *mesh, int32_t n, const tlfe_constraint *cons_dev, const double *u_dev,
                              const double *v_dev, double *out_dev, void *stream);

/* Launch-schedule autotuner (no counterpart in the paper; a property of this
 * GPU implementation). For every element block it times the force, operator
 * (when v_dev is given) and adjoint (when v_dev is given) kernels on the
 * caller's state over the resident CTA sizes (4, 2, 1 warps) and both tile
 * assignments (interleaved; contiguous runs per warp), writing into scratch
 * arrays, and keeps the fastest schedule for later calls with the same
 * material mode (velocity given or not); with v_dev on an FP32 mesh it also
 * tunes the one-pass force + operator product of tlfe_force_matvec and keeps
 * that pass only if it measures faster than the two passes. Results of later
 * calls are unchanged up to the order of floating-point additions in the
 * scatter.
 * u_dev: device double [n_nodes][3]; udot_dev, v_dev: device [n_nodes][3] in
 * the mesh dtype, or NULL. Allocates and frees scratch; synchronises `stream`.
 * Optional: without it, the schedule comes from the occupancy API. */
tlfe_status tlfe_autotune(tlfe_mesh *mesh, const double *u_dev, const void *udot_dev, const void *v_dev,
                          void *stream);

/* Replace the per-element Lame parameters (mu_e, lambda_e) of every element
 * (device double [n_elem][2], global element order); later calls use them in
 * place of the body materials' (mu, lambda). The first call on a handle created
 * without elem_mu_lambda allocates the per-element copy. Stream-ordered; the
 * caller's array is not kept. */
tlfe_status tlfe_set_elem_mu_lambda(tlfe_mesh *mesh, const double *mu_lambda_dev, void *stream);

/* Vector-Jacobian products of f_int against a cotangent r:
 *   g_u = K_t^T r,   g_udot = C^T r,
 *   g_mu_lambda[e] = (r . d f / d mu_e, r . d f / d lambda_e)
 * u_dev: device double [n_nodes][3]; udot_dev, cot_dev, g_u_dev, g_udot_dev:
 * device [n_nodes][3] in the mesh dtype;
 * g_mu_lambda_dev: device double [n_elem][2]. Any output may be NULL (not
 * computed); non-NULL outputs are overwritten. */
tlfe_status tlfe_vjp(tlfe_mesh *mesh, const void *u_dev, const void *udot_dev, const void *cot_dev,
                     void *g_u_dev, void *g_udot_dev, double *g_mu_lambda_dev, void *stream);

/* Backward-Euler step (Sec. 7, Eqs. step_map_velocity_level and residual):
 * find v with
 *   g(v) = M/h (v - v_n) + f_int(u_n + h v, v) - f_ff - f_ext
 *          [+ h C_q^T (lambda + rho c)] = 0,
 * f_ff_i = rho v_i b0 (Eq. virtual_work_force_field_uniform), f_ext the
 * optional applied load (f_ext_dev; dead load over the step), by inexact
 * Newton: each iteration solves (M/h + h K^e + C) dv = -g by Jacobi-PCG with
 * per-body scalars (all bodies advance together, each stops on its own), and
 * stops when ||g_b|| <= newton_rtol ||g_b(v_n)|| for every body b. The residual
 * and the update of v are FP64; the operator products and the CG vectors run
 * in the mesh precision, and the CG dots are summed per chunk in FP64 (an
 * FP32 mesh forms each thread's share in double-float arithmetic, about 44
 * significant bits). Nodes with fixed_dev[k] = 1 are clamped (v = 0).
 * The whole step is one CUDA graph with conditional WHILE nodes (built on the
 * first call, replayed afterwards).
 * With constraints (n_cons > 0) the step is the augmented-Lagrangian iteration
 * of Sec. 7: Newton solves of g(v, lambda) = 0, whose CG matrix adds the
 * Gauss-Newton term h^2 rho C_q^T C_q (the curvature terms of App. B.2 are left
 * out), alternate with lambda += rho c(q(v)) (Eq. alm_multiplier_update) until
 * ||c|| <= alm_tol or max_outer updates; the Newton solves after the first
 * start from the previous v and stop relative to the step's first residual.
 * The step works on row-normalised constraints c^_k = w_k c_k (Eqs. row_weights,
 * rev_normalized): w_k = 1 / sqrt(|a_0|^2 + |b_0|^2) for a DP1 row, with a_0 and
 * b_0 its two directions in the reference configuration, and w_k = 1 for CD,
 * DIST and DP2 rows. lambda_dev holds the multipliers of the normalised rows
 * and c_norm is ||c^||; tlfe_constraint_eval / _j / _jt return raw rows.
 * Constraints may couple bodies: the whole mesh is then solved as one system
 * (one convergence test). */
typedef struct {
    double h;
    double gravity[3];
    double newton_rtol;
    double cg_rtol;
    int32_t max_newton;
    int32_t max_cg;
    const uint8_t *fixed_dev;  /* device [n_nodes], or NULL */
    int32_t use_graph;         /* 1 = CUDA graph with conditional nodes, 0 = host-driven loop */
    const double *f_ext_dev;   /* device double [n_nodes][3] applied load of the step (Sec. 4:
                                  point loads, tractions), or NULL; read at every call */
    /* augmented-Lagrangian constraints (Sec. 7); n_cons = 0 for none */
    int32_t n_cons;
    const tlfe_constraint *cons_dev;  /* device [n_cons] */
    double rho;                /* penalty rho > 0 */
    double alm_tol;            /* stop when ||c^(q(v))||_2 <= alm_tol (normalised rows) */
    int32_t max_outer;         /* multiplier updates at most */
    double *lambda_dev;        /* device double [n_cons], multipliers of the normalised rows, in/out */
} tlfe_step_params;

typedef struct {
    int32_t newton_iters;      /* max over bodies */
    int32_t cg_iters;          /* total CG iterations run by the step */
    int32_t status;            /* tlfe_status of the step */
    int32_t n_bodies_converged;
    double rel_residual;       /* max over bodies of ||g_b|| / ||g_b(v_n)|| */
    int32_t outer_iters;       /* multiplier updates (constraints) */
    double c_norm;             /* ||c^(q(v))||_2 at return (normalised rows) */
} tlfe_step_report;

/* u_n_dev, v_n_dev, v_out_dev: device double [n_nodes][3]. report_host is
 * written before return. Synchronises `stream`. */
tlfe_status tlfe_newton_step(tlfe_mesh *mesh, const double *u_n_dev, const double *v_n_dev,
                             const tlfe_step_params *params, double *v_out_dev,
                             tlfe_step_report *report_host, void *stream);

/* Per-body Euclidean norms of a node array (the deterministic FP64 reduction
 * the Newton step uses for its residual and CG tests, Sec. 7):
 *   out_dev[b] = sqrt(sum over the nodes k of body b of |x_k|^2)
 * x_dev: device double [n_nodes][3]; out_dev: device double [n_bodies].
 * Every body must own one contiguous node range and share no node with another
 * body (TLFE_E_UNSUPPORTED otherwise). The first call (or the first Newton
 * step) allocates the reduction workspace of the handle. Stream-ordered; the
 * result does not depend on the launch configuration. */
tlfe_status tlfe_body_norms(tlfe_mesh *mesh, const double *x_dev, double *out_dev, void *stream);

/* Euclidean norm of a device vector, for callers that cannot allocate device
 * memory: a process that has reserved its whole device budget up front (a
 * real-time or embedded control loop, a host application that hands out all
 * GPU memory from its own pool) or code that must not call cudaMalloc on its
 * hot path because it synchronises the device and can fail at run time. The
 * paper has no counterpart; this is the same deterministic chunked FP64
 * reduction as tlfe_body_norms, without a mesh handle or workspace.
 *   *out_dev = sqrt(sum_k x_dev[k]^2),  k < n
 * x_dev: device double [n]; out_dev: device double [1]. n must be at most
 * 4096 * 4096 = 16,777,216 (TLFE_E_INVALID beyond, with a message naming the
 * limit): the partial sums live in a fixed 32 KiB array in device memory that
 * every GPU loading the library holds until the process exits.
 * Allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 * Each device that loads the library has its own copy of the array. The first
 * call on a device looks up that copy's device address, once per device and
 * with that device current, so make that first call before any stream
 * capture. Every call on one device uses that device's copy and leaves its
 * partial sums there: calls that overlap on the same device (different
 * streams) race, so order them on one stream; calls on different devices do
 * not interfere. The looked-up address lasts as long as the device's context:
 * after cudaDeviceReset on that device, restart the process before calling
 * this entry point again. */
tlfe_status tlfe_norm_noalloc(const double *x_dev, int64_t n, double *out_dev, void *stream);

/* Diagnostic of the timeout path of device-side waits (no counterpart in the
 * paper). The element kernels wait for their bulk copies with a bounded number
 * of mbarrier try_wait rounds and, when a copy never lands, record the fact in
 * the mesh's status word and return instead of hanging. This call runs that
 * wait on an mbarrier that expects 16 bytes no copy will deliver, for
 * spin_limit rounds (1 .. 2^20; each round may pause the thread for a
 * hardware-chosen time slice), then records the timeout the same way: the next
 * tlfe_sync returns TLFE_E_TIMEOUT and clears the status, and the mesh and
 * the CUDA context stay usable. Stream-ordered; no fault, no trap. */
tlfe_status tlfe_selftest_wait_timeout(tlfe_mesh *mesh, int64_t spin_limit, void *stream);

/* Node rows of a [n_nodes][3] array to and from a compact buffer, for the
 * interface exchange of one body split across GPUs (its elements in slabs,
 * the nodes of the slab interfaces duplicated): after each operator
 * application the ranks sum their partial rows of the interface nodes through
 * one compact buffer (Sec. 4.3 assembly across the split).
 *   tlfe_gather_nodes : out[o(k)][c] = x[idx[k]][c], o(k) = out_idx[k], or k
 *                       when out_idx is NULL; rows 0 .. n_out_clear - 1 of
 *                       out are zeroed first (0: none)
 *   tlfe_scatter_nodes: x[idx[k]][c] = in[i(k)][c], i(k) = in_idx[k], or k
 * k < n, c < 3; float (TLFE_FP32) or double (TLFE_FP64) arrays; index arrays
 * device int32 [n] (a destination row listed twice gets one of the values).
 * Device pointers; stream-ordered; no mesh handle. */
tlfe_status tlfe_gather_nodes(int32_t precision, const void *x_dev, const int32_t *idx_dev, int32_t n,
                              void *out_dev, const int32_t *out_idx_dev, int32_t n_out_clear, void *stream);
tlfe_status tlfe_scatter_nodes(int32_t precision, const void *in_dev, const int32_t *in_idx_dev,
                               const int32_t *idx_dev, int32_t n, void *x_dev, void *stream);

/* The CG operator of the Newton step (Sec. 2.2 Newton matrix, Sec. 7; App. C
 * tangent blocks): y = a_M M v + a_K K^e(u) v + a_C C(u) v, the symmetric
 * part of the operator of tlfe_tangent_matvec (the viscous stiffness K^v of
 * the Kelvin-Voigt law left out), whose diagonal tlfe_jacobi_diag returns.
 * Arguments, layouts and errors as tlfe_tangent_matvec. */
tlfe_status tlfe_newton_operator(tlfe_mesh *mesh, const void *u_dev, const void *udot_dev,
                                 const void *v_dev, double a_M, double a_K, double a_C,
                                 void *y_dev, void *stream);

/* Backward-Euler step of one body split across GPUs (Sec. 7, Eqs.
 * step_map_velocity_level and residual; the inexact Newton / Jacobi-PCG
 * iteration of tlfe_newton_step). Each rank holds a mesh of its slab of
 * elements and every node they touch, so interface nodes sit on two ranks.
 * The caller drives the iteration on the host:
 *   residual  tlfe_split_prep, then f = tlfe_internal_force(u, v) and
 *             y = tlfe_tangent_matvec(a_M = 1/h, a_K = a_C = 0) on w, then
 *             tlfe_split_residual; the interface rows of g summed over the
 *             ranks; ||g||^2 = tlfe_split_dot(g, g), all-reduced
 *   CG        D = tlfe_jacobi_diag(1/h, h, 1), interface-summed, then
 *             tlfe_split_cg_dinv and tlfe_split_cg_start (r.z, r.r, all-reduced);
 *             per iteration q = tlfe_newton_operator(1/h, h, 1) on p,
 *             interface-summed, tlfe_split_cg_pq (p.q, all-reduced),
 *             alpha = r.z / p.q, tlfe_split_cg_update (the new r.z and r.r,
 *             all-reduced), beta = r.z(new) / r.z, tlfe_split_cg_direction
 *   update    tlfe_split_velocity(v, add_x = 1)
 * so that per CG iteration the ranks exchange one compact interface buffer
 * and all-reduce three FP64 scalars. Every sum over rows counts only the rows
 * with own[k] = 1 (each interface node is owned by exactly one rank), in FP64
 * and in a fixed order: a chunk partial of 4096 values per CTA into work_dev,
 * then the partials in order into dots_dev (deterministic). The caller
 * all-reduces dots_dev and reads the sums on the host.
 * Clamped rows (fixed[k] = 1) are projected out of g, r, z, p, q and v.
 * x, r, p, q, dinv: device [n_rows][3] in `precision` (the operator mesh's);
 * every other vector is device double [n_rows][3]. All pointers are
 * caller-owned device memory; no call allocates. Stream-ordered. */
typedef struct {
    int32_t precision;       /* TLFE_FP32 / TLFE_FP64: dtype of x, r, p, q, dinv */
    int32_t n_rows;          /* node rows of this rank's share (>= 0) */
    const uint8_t *fixed;    /* device [n_rows], 1 = clamped node, or NULL (none) */
    const uint8_t *own;      /* device [n_rows], 1 = row counted in sums, or NULL (all) */
    void *x, *r, *p, *q, *dinv;
    double *work;            /* device, tlfe_split_work_doubles(n_rows) doubles */
    double *dots;            /* device double [2]: partial sums of the last call */
} tlfe_split_cg;

/* Doubles of work_dev for a share of n_rows node rows. */
int64_t tlfe_split_work_doubles(int64_t n_rows);
/* u_out = u_n + h v; w_out = v - v_n - h b0, b0 = gravity_host[3] (so that
 * M/h w = M/h (v - v_n) - f_ff with f_ff = M b0, Sec. 4.2); v_op_out, when not
 * NULL, receives v in `precision` (the operator mesh's udot). */
tlfe_status tlfe_split_prep(const tlfe_split_cg *c, double h, const double *gravity_host,
                            const double *u_n, const double *v_n, const double *v, double *u_out,
                            double *w_out, void *v_op_out, void *stream);
/* g = f + y with the clamped rows zeroed (this rank's partial residual). */
tlfe_status tlfe_split_residual(const tlfe_split_cg *c, const double *f, const double *y, double *g,
                                void *stream);
/* v_out = v_base (+ x when add_x), clamped rows zeroed; v_out may be v_base. */
tlfe_status tlfe_split_velocity(const tlfe_split_cg *c, const double *v_base, int32_t add_x,
                                double *v_out, void *stream);
/* dots[0] = sum over owned rows of a . b (double arrays). */
tlfe_status tlfe_split_dot(const tlfe_split_cg *c, const double *a, const double *b, void *stream);
/* dinv = 1 / D on free rows with D != 0, else 0 (D in `precision`). */
tlfe_status tlfe_split_cg_dinv(const tlfe_split_cg *c, const void *D, void *stream);
/* x = 0, r = -g (clamped rows 0), p = dinv r; dots = (r . dinv r, r . r). */
tlfe_status tlfe_split_cg_start(const tlfe_split_cg *c, const double *g, void *stream);
/* q: clamped rows zeroed; dots[0] = p . q. */
tlfe_status tlfe_split_cg_pq(const tlfe_split_cg *c, void *stream);
/* x += alpha p, r -= alpha q; dots = (r . dinv r, r . r). */
tlfe_status tlfe_split_cg_update(const tlfe_split_cg *c, double alpha, void *stream);
/* p = dinv r + beta p. */
tlfe_status tlfe_split_cg_direction(const tlfe_split_cg *c, double beta, void *stream);

/* Arithmetic peak probe (no counterpart in the paper; the denominator of the
 * element kernels' ALU roofline): enqueues one kernel of ctas_per_sm CTAs of
 * 256 threads per SM in which every thread runs 16 independent fused
 * multiply-add chains for `iters` rounds, in FP32 (precision = TLFE_FP32) or
 * FP64 (TLFE_FP64). *flop_host receives the launch's FLOP count (2 per FMA);
 * time the launch with events on `stream` for the rate. out_dev: device
 * buffer of at least 2 values of that precision (receives a checksum).
 * ctas_per_sm in [1, 32], iters in [1, 2^32]. Stream-ordered. */
tlfe_status tlfe_peak_probe(int32_t precision, int32_t ctas_per_sm, int64_t iters, void *out_dev,
                            double *flop_host, void *stream);

/* Thread-local text of the last error (never NULL). */
const char *tlfe_last_error(void);

/* Library version string. */
const char *tlfe_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TLFE_H */
