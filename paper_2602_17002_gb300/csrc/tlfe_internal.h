// Internal structures shared by the translation units of libtlfe.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "tlfe.h"
#include "tlfe_math.cuh"

namespace tlfe {

// OP_FM: internal force and operator product of one state in one pass
// (outputs f and y; the gather, kinematics and stress state shared)
enum { OP_FORCE = 0, OP_MATVEC = 1, OP_VJP = 2, OP_DIAG = 3, OP_FM = 4 };
// status word: counts of device-side events, read and cleared by tlfe_sync;
// ST_BOUNDS counts table indices found out of range (bounds-checked build)
enum { ST_INVERTED = 0, ST_NONFINITE = 1, ST_TIMEOUT = 2, ST_BOUNDS = 3, ST_COUNT = 4 };
// material modes of an element launch: the law and the viscous term fixed at
// compile time, or both read per element (MAT_ANY)
enum { MAT_ANY = 0, MAT_NH = 1, MAT_NH_KV = 2, MAT_SVK = 3, MAT_SVK_KV = 4 };

constexpr int TILE = 32;     // elements per tile = lanes of one warp
constexpr int AFF_ROWS = 10;  // affine record rows per tile: J^{-1} (9, row-major), det J
// affine Q27 blocks run the warp-per-element kernels (one warp per element,
// lanes over points then nodes); every other block runs one thread per element
__host__ __device__ inline bool wpe_path(int et, bool aff) { return et == ET_Q27 && aff; }

// values per node held in a warp's shared-memory patch: inputs (u, udot
// [, v or cotangent]) then outputs (one array, two for the adjoint)
__host__ __device__ constexpr int op_in_fields(int op) { return (op == OP_MATVEC || op == OP_VJP || op == OP_FM) ? 9 : 6; }
__host__ __device__ constexpr int op_nf(int op) { return op_in_fields(op) + ((op == OP_VJP || op == OP_FM) ? 6 : 3); }

// Everything an element kernel needs about one block and one call.
template <typename R> struct KParams {
    // block layout (AoSoA tiles of 32 elements, see create_mesh)
    int tile_begin, tile_end;
    int umax;                   // max unique nodes of a tile (shared-memory patch records)
    const int32_t *tnode_off;   // [n_tiles + 1] offsets into tnodes
    const int32_t *tnodes;      // node list of each tile: its unique global node ids, in patch order
    const uint16_t *lidx;       // [n_tiles][npe][32] index of (elem, node) into the tile's list
    // per-tile metadata records of meta_bytes each (16-byte multiple):
    //   int32 U, int32 first partial position (sorted scatter), 2 x pad |
    //   int32 eid[32] | int32 node id[umaxp] | u16 lidx[npe][32] |
    //   u16 position[npe * 32] (slot i * 32 + lane -> its place in the node-grouped order) |
    //   u16 node offsets[U + 1] into that order (padded)
    const unsigned char *meta;
    int meta_bytes, umaxp;
    const int32_t *eid;         // [n_tiles][32] global element id, -1 for padding lanes
    const int32_t *conn;        // [n_elem][npe] global node ids, block element order (warp-per-element path)
    int elem_base;              // global id of the block's first element
    const R *slab;              // [n_tiles][nq][3 npe + 1][32]: h_i components, then w_q J_p
    const R *aff;               // affine path: [n_tiles][10][32] J^{-1} (row-major) and det J; nullptr = slab path
    const int32_t *emat;        // [n_tiles][32] material index, or nullptr (uniform mat0)
    const R *elam;              // [n_tiles][2][32] per-element (mu, lam), or nullptr
    const R *evol;              // [n_tiles][32] element volume (affine mass)
    // materials
    Mat<R> mat0;
    const Mat<R> *mats;
    // state and outputs ([n_nodes][3] arrays)
    const double *u;            // displacement, always FP64 (see Rec in k_elem.cuh)
    const R *ud, *v;
    R *out0, *out1;
    double *gth;                // [n_elem][2] (VJP parameter gradient)
    R aM, aK, aC;
    int sym_only;
    int mass_only;              // operator product with a_K = a_C = 0: no quadrature loop, no slab stream
    int rmw_scatter;            // 1: plain read-add-write (colour passes), 0: atomics
    // sorted scatter (part0 != nullptr): per-node tile sums are stored to
    // part{0,1}[position * 3 + c] instead of being added, with position
    // part_base + toff[t] + k for unique node k of tile t (tile kernels: the
    // record header holds part_base + toff[t]) or part_base + slot * 27 + n
    // (warp-per-element kernels)
    R *part0, *part1;
    int64_t part_base;
    int visc;                   // udot given and material damped somewhere in the block
    int mat_mode;               // MAT_* (compile-time material of the launched kernel)
    int tile_chunk;             // 1: each warp takes a contiguous run of tiles; 0: interleaved
    int *status;                // [ST_COUNT]
    // extents of the arrays the tables index, for the bounds-checked build
    // (TLFE_BOUNDS_CHECK): node arrays, parameter gradient, partial sums, materials
    int n_nodes, n_elem_total, n_mats, n_elem_block;
    int64_t n_part;
};

// Bounds-checked build (compiled with TLFE_BOUNDS_CHECK): an index read from a
// device table is checked against the extent of the array it addresses; an
// index out of range is counted in the status word (ST_BOUNDS, reported by
// tlfe_sync) and clamped into the array, so that the access stays in bounds.
// The normal build compiles the checks away.
__device__ __forceinline__ int64_t bounds_clamp(int64_t x, int64_t lim, int *status)
{
#ifdef TLFE_BOUNDS_CHECK
    if (x < 0 || x >= lim) {
        atomicAdd(status + ST_BOUNDS, 1);
        return x < 0 ? 0 : (lim > 0 ? lim - 1 : 0);
    }
#endif
    return x;
}
// whether an index is in range (always true in the normal build); counts misses
__device__ __forceinline__ bool bounds_ok(int64_t x, int64_t lim, int *status)
{
#ifdef TLFE_BOUNDS_CHECK
    if (x < 0 || x >= lim) {
        atomicAdd(status + ST_BOUNDS, 1);
        return false;
    }
#endif
    return true;
}

// element-kernel launcher for one op and precision, dispatching on (element
// type, nq) and on the path (affine when p.aff is set, else the slab);
// grid = number of CTAs of wpb warps each, grid-striding over tiles.
// Defined in k_elem.cuh and instantiated in k_force.cu / k_matvec.cu /
// k_vjp.cu / k_diag.cu.
template <int OP, typename R>
cudaError_t launch_op(int et, int nq, const KParams<R> &p, int grid, int wpb, cudaStream_t s);

// warps per SM the kernel of (op, et, nq, precision, path) can keep resident
// for a block whose tiles hold at most `umax` unique nodes
// (CTA sizes of 1, 2 and 4 warps are tried; *wpb receives the best one)
template <int OP, typename R>
int occupancy_op(int et, int nq, bool aff, int mat, int umax, int meta_bytes, int *wpb, std::string *why);

// set-up kernels
cudaError_t launch_precompute(int et, int nq, int precision, int n_tiles, const int32_t *eid,
                              const int32_t *conn_elem, int elem_base, const double *X, void *slab,
                              void *evol, int *affine_flag, int *status, cudaStream_t s);
cudaError_t launch_precompute_affine(int et, int precision, int n_tiles, const int32_t *eid,
                                     const int32_t *conn_elem, int elem_base, const double *X, void *aff,
                                     void *evol, int *affine_flag, int *status, cudaStream_t s);
cudaError_t launch_set_elam(int precision, int n_tiles, const int32_t *eid, const double *src, void *elam,
                            cudaStream_t s);
cudaError_t launch_color_round(int n_elem, int npe, const int32_t *conn, const int32_t *inc_off,
                               const int32_t *inc, const int32_t *elem_local_to_block,
                               uint64_t seed, int elem_base, int32_t *color, int *n_left,
                               int *overflow, cudaStream_t s);

// ---- constraint primitives (constraints.cu) ----
constexpr int CON_MAXN = 27;  // nodes of the largest element (Q27)
constexpr int CON_MAXB = 16;  // element blocks a constraint set can refer to
struct ConBlocks {            // block table passed to the kernels by value
    int n;
    int et[CON_MAXB], base[CON_MAXB], ne[CON_MAXB];
    const int32_t *conn[CON_MAXB];
};
cudaError_t con_prepare(const ConBlocks &bt, int n, const tlfe_constraint *cons, double *sh, int32_t *nd, int *bad,
                        cudaStream_t s);
cudaError_t con_eval(int n, const tlfe_constraint *cons, const double *sh, const int32_t *nd, const double *X,
                     const double *u, const double *wrow, double *c, double *gp, cudaStream_t s);
cudaError_t con_row_weights(int n, const tlfe_constraint *cons, const double *sh, const int32_t *nd, const double *X,
                            double *wrow, cudaStream_t s);
template <typename R>
cudaError_t con_jt(int n, const double *sh, const int32_t *nd, const double *gp, const double *w, double scale, R *f,
                   cudaStream_t s);
template <typename V>
cudaError_t con_j(int n, const double *sh, const int32_t *nd, const double *gp, const V *v, double *out,
                  cudaStream_t s);
template <typename R>
cudaError_t con_diag(int n, const double *sh, const int32_t *nd, const double *gp, double alpha, R *D, cudaStream_t s);
cudaError_t con_weights(int n, const double *lam, const double *c, double rho, double h, double *w, cudaStream_t s);
cudaError_t con_lam_update(int n, double *lam, const double *c, double rho, cudaStream_t s);

}  // namespace tlfe
