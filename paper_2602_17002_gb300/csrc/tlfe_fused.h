// Host-visible part of the fused (one launch per operation) element kernels:
// the launch's parameter table and the launch helpers (k_fused.cuh).
#pragma once

#include "tlfe_internal.h"

namespace tlfe {

constexpr int FUSED_MAXP = 56;  // passes one fused launch can cover (the table lives in kernel parameters)

// element type / quadrature codes of the fused kernels
enum { FK_T4Q1 = 0, FK_T10Q4 = 1, FK_T10Q5 = 2, FK_H8Q8 = 3, FK_N = 4 };
constexpr int MAT_N = 5;  // MAT_ANY .. MAT_SVK_KV

__host__ __device__ inline int fused_code(int et, int nq)
{
    if (et == ET_T4 && nq == 1) return FK_T4Q1;
    if (et == ET_T10 && nq == 4) return FK_T10Q4;
    if (et == ET_T10 && nq == 5) return FK_T10Q5;
    if (et == ET_H8 && nq == 8) return FK_H8Q8;
    return -1;
}

template <typename R> struct FusedArgs {
    int n_items;
    const int4 *items;     // (pass, first tile, end tile, 0) in the order warps take them
    int *counter;          // next item to take; zero before the launch
    int wreg;              // bytes of one warp's shared-memory region
    int kind[FUSED_MAXP];  // fused_code * MAT_N + material mode, per pass
    KParams<R> pass[FUSED_MAXP];
};

// defined in k_fused.cuh, instantiated for (OP_FORCE, float) in
// k_fused_force.cu and (OP_MATVEC, float) in k_fused_matvec.cu
template <typename R, int OP> size_t fused_warp_region(int code, int umax, int meta_bytes);
template <int OP, typename R> int occupancy_fused(size_t wreg, int *wpb_io);
template <int OP, typename R> cudaError_t launch_fused(const FusedArgs<R> &a, int grid, int wpb, cudaStream_t s);

}  // namespace tlfe
