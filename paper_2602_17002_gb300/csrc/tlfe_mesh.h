// Host-side mesh handle of libtlfe.
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "tlfe_internal.h"

namespace tlfe {

struct NewtonState;  // newton.cu

// One element block as stored on the device.
struct LaunchSched {
    int resident = 0;   // resident warps per SM at wpb warps per CTA (0: not resident)
    int wpb = 0;        // warps per CTA
    int chunk = 0;      // 1: contiguous tile runs per warp; 0: interleaved
    bool tuned = false; // chosen by measurement
};

struct BlockStore {
    int et = 0, nq = 0, npe = 0, n_elem = 0, elem_base = 0, n_tiles = 0, umax = 0;
    int n_colors = 0;
    bool affine = false;             // every element affine (Sec. 6, affine case)
    bool use_affine = false;         // kernels run on the affine path (J^{-1}, det J per element)
    int model = -1;                  // elastic law shared by every element of the block, or -1
    bool visc = false;
    int uniform_body = 0;            // body id when every element shares it, else -1
    int64_t n_unique = 0;            // sum over tiles of the unique node count
    int64_t patch_loads = 0;         // quarter-warp node-patch loads of one pass over the tiles (per
    int64_t patch_passes = 0;        // element-local node) and the shared-memory passes they take
    // passes: tile range [color_tile_off[c], color_tile_off[c + 1]) of pass c,
    // one per (colour in colour mode,) elastic law; the law and whether any
    // element of the pass is damped
    std::vector<int> color_tile_off;
    std::vector<int> pass_model;
    std::vector<bool> pass_visc;
    std::vector<int32_t> colors;     // colour of each block element (colour mode)
    int32_t *d_eid = nullptr, *d_toff = nullptr, *d_tnodes = nullptr, *d_emat = nullptr;
    uint16_t *d_lidx = nullptr;
    unsigned char *d_meta = nullptr;  // per-tile metadata records
    int meta_bytes = 0, meta_umaxp = 0;
    void *d_slab = nullptr, *d_evol = nullptr, *d_elam = nullptr;
    void *d_aff = nullptr;           // [n_tiles][10][32] J^{-1}, det J (affine path)
    int32_t *d_conn = nullptr;       // [n_elem][npe] global node ids (block element order)
    int64_t part_base = 0;           // sorted scatter: first partial-sum position of the block
};

// One persistent launch per operation over the passes of an FP32 mesh (atomic
// or sorted scatter) whose blocks run the affine tile kernels: the work items
// (pass, first tile, end tile) in the order warps take them, and per fused op
// (force, operator product) its launch schedule and warp-region size.
struct FusedPlan {
    std::vector<std::pair<int, int>> passes;  // (block, pass) covered, in table order
    std::vector<bool> covered;                // per block: its passes run in the fused launch
    int n_items = 0;
    int4 *d_items = nullptr;
    int *d_counter = nullptr;                 // one counter per fused op
    LaunchSched sched[2];                     // [0] force, [1] operator product
    size_t wreg[2] = {0, 0};
    bool on[2] = {true, true};                // fused (true) or per-pass launches, per op
};

struct OpGraph;    // graph.cu: the captured force + operator-product call
struct HostStage;  // hoststep.cu: staging buffers and copy streams of tlfe_step_host

}  // namespace tlfe

struct tlfe_mesh {
    int device = 0, n_sm = 0;
    int precision = TLFE_FP32, scatter = TLFE_SCATTER_ATOMIC;
    int n_nodes = 0, n_elem = 0, n_bodies = 0;
    int64_t n_qp = 0;
    int64_t device_bytes = 0;
    std::vector<tlfe::BlockStore> blocks;
    std::vector<tlfe_material> h_mats;
    tlfe::Mat<float> *d_mats_f = nullptr;
    tlfe::Mat<double> *d_mats_d = nullptr;
    int *d_status = nullptr;
    double *d_X = nullptr;
    void *d_stage = nullptr;        // staging buffers of tlfe_internal_force_host
    void *d_scratch_vjp = nullptr;  // stand-in outputs of tlfe_vjp
    tlfe::NewtonState *newton = nullptr;
    // host copy of the creation description (the Newton step builds an FP64
    // twin of an FP32 mesh from it) and the node -> body map
    std::vector<double> h_X;
    std::vector<std::vector<int32_t>> h_conn, h_body;
    std::vector<tlfe_block> h_blocks;
    std::vector<double> h_elam;
    uint64_t color_seed = 0;
    int element_path = TLFE_PATH_AUTO;
    int patch_layout = TLFE_PATCH_BANKED;
    std::vector<int32_t> node_body;  // body of each node (-1: in no element)
    std::vector<void *> allocs;
    // launch schedule of one (op, block, material mode, precision): resident
    // warps per SM at `wpb` warps per CTA, and the tile assignment; filled from
    // the occupancy API on first use, replaced by measurement in tlfe_autotune
    std::map<std::tuple<int, int, int, int>, tlfe::LaunchSched> sched;
    // sorted scatter: the node of every partial-sum position (-1: unused),
    // filled block by block at creation; its transpose (positions of node n
    // in ascending order: part_pos[part_ptr[n] .. part_ptr[n + 1])) and the
    // two partial buffers [2][n_part][3] in the mesh precision
    std::vector<int32_t> h_part_node;
    int64_t n_part = 0;
    int64_t *d_part_ptr = nullptr;
    int32_t *d_part_pos = nullptr;
    void *d_part = nullptr;
    // fused launch plan (nullptr when the mesh has fewer than two passes the
    // fused kernels cover, or is FP64 or coloured) and the launch mode
    tlfe::FusedPlan *fused = nullptr;
    int launch_mode = TLFE_LAUNCH_AUTO;
    tlfe::OpGraph *fm_graph = nullptr;
    int sched_gen = 0;  // bumped whenever launch schedules, mode or block parameters change
    tlfe::HostStage *host_stage = nullptr;
    // the force and the operator product of one state as one fused pass
    // (OP_FM) where the mesh allows it; tlfe_autotune sets it by measurement
    int fm_on = 1;
    // scratch of the standalone constraint calls (tlfe_constraint_eval / _j /
    // _jt): point data for con_cap constraints, grown on demand and kept
    // until the handle is destroyed
    int con_cap = 0;
    double *d_con_sh = nullptr, *d_con_gp = nullptr, *d_con_c = nullptr;
    int32_t *d_con_nd = nullptr;
    int *d_con_bad = nullptr;
};

namespace tlfe {

// NVTX range named after the C entry point for the duration of the call, so
// that profilers and timelines attribute the kernels a call launches to it
// (free when no tool is attached)
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
#define TLFE_TRACE(name) tlfe::TraceRange tlfe_trace_range_(name)

tlfe_status fail(tlfe_status st, const std::string &msg);
// force and operator product of one state (tlfe_force_matvec, tlfe_step_host):
// one fused pass where fm_eligible, else the two passes; the argument checks
// of tlfe_internal_force and tlfe_tangent_matvec together
bool fm_eligible(const tlfe_mesh *m);
tlfe_status force_matvec_op(tlfe_mesh *m, const void *u, const void *ud, const void *v, double aM, double aK,
                            double aC, void *f, void *y, cudaStream_t s);
tlfe_status check_force_matvec(tlfe_mesh *m, const void *u, const void *v, const void *f, const void *y, double aM,
                               double aK, double aC);
void destroy_graphs(tlfe_mesh *m);      // graph.cu
void destroy_host_stage(tlfe_mesh *m);  // hoststep.cu
tlfe_status cuda_fail(cudaError_t e, const char *where);
void *dalloc(tlfe_mesh *m, size_t bytes, cudaError_t *err);
void destroy_newton(tlfe_mesh *m);
tlfe_mesh *newton_twin(tlfe_mesh *m);  // FP64 twin of an FP32 mesh built by the Newton step, or nullptr
ConBlocks con_blocks(const tlfe_mesh *m);  // n = -1 when the mesh has more blocks than a constraint set supports

template <int OP, typename R>
tlfe_status run_op(tlfe_mesh *m, const void *u, const void *ud, const void *v, void *out0, void *out1,
                   double *gth, double aM, double aK, double aC, int sym_only, cudaStream_t s);

}  // namespace tlfe
