// tlfe_step_host / tlfe_step_host_wait: the element operations of one state
// on HOST buffers, with the transfers overlapped with the computation.
//
// The handle keeps two sets of device staging buffers and two copy streams
// of its own (host-to-device, device-to-host). Call k uses set k mod 2: its
// inputs are copied in on the first copy stream as soon as the last
// computation that read that set has ended; the operations run on the
// caller's stream once the inputs have arrived (and once the set's outputs
// from two calls back have been copied out); each output goes back on the
// second copy stream as soon as the operation that writes it has ended. So
// call k + 1's inputs arrive while call k computes, and call k's outputs
// leave while call k + 1 computes.
#include <cuda_runtime.h>

#include "tlfe_mesh.h"

namespace tlfe {

struct HostStage {
    size_t nu = 0, nb = 0, ng = 0;           // bytes: FP64 node array, mesh-precision node array, g_theta
    char *d_in[2] = {nullptr, nullptr};      // per set: u | udot | v | cot
    char *d_out[2] = {nullptr, nullptr};     // per set: f | y | g_u | g_udot | g_theta
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t in_ready[2] = {}, comp_done[2] = {}, out_done[2] = {}, op_done[2][3] = {};
    bool used[2] = {false, false};
    int64_t calls = 0;
};

void destroy_host_stage(tlfe_mesh *m)
{
    HostStage *h = m->host_stage;
    if (!h) return;
    if (h->h2d) cudaStreamSynchronize(h->h2d);
    if (h->d2h) cudaStreamSynchronize(h->d2h);
    for (int b = 0; b < 2; ++b) {
        cudaEvent_t evs[6] = {h->in_ready[b], h->comp_done[b], h->out_done[b], h->op_done[b][0], h->op_done[b][1],
                              h->op_done[b][2]};
        for (cudaEvent_t e : evs)
            if (e) cudaEventDestroy(e);
    }
    if (h->h2d) cudaStreamDestroy(h->h2d);
    if (h->d2h) cudaStreamDestroy(h->d2h);
    delete h;  // the staging buffers are mesh allocations, freed with the handle
    m->host_stage = nullptr;
}

static tlfe_status make_stage(tlfe_mesh *m)
{
    HostStage *h = new HostStage();
    m->host_stage = h;
    const size_t rs = m->precision == TLFE_FP32 ? 4 : 8;
    h->nu = (size_t)3 * m->n_nodes * 8;
    h->nb = (size_t)3 * m->n_nodes * rs;
    h->ng = (size_t)2 * m->n_elem * 8;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        h->d_in[b] = (char *)dalloc(m, h->nu + 3 * h->nb, &e);
        if (e == cudaSuccess) h->d_out[b] = (char *)dalloc(m, 4 * h->nb + h->ng, &e);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->d2h, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        cudaEvent_t *evs[6] = {&h->in_ready[b], &h->comp_done[b], &h->out_done[b], &h->op_done[b][0],
                               &h->op_done[b][1], &h->op_done[b][2]};
        for (cudaEvent_t *ev : evs)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        destroy_host_stage(m);
        return cuda_fail(e, "tlfe_step_host: staging set-up");
    }
    return TLFE_OK;
}

}  // namespace tlfe

using namespace tlfe;

#define CKH(call)                                                   \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return tlfe::cuda_fail(e_, #call);   \
    } while (0)

extern "C" tlfe_status tlfe_step_host(tlfe_mesh *m, const tlfe_host_step *a, void *stream)
{
    TLFE_TRACE("tlfe_step_host");
    if (!m || !a || !a->u_host) return fail(TLFE_E_INVALID, "tlfe_step_host: mesh, args and u_host are required");
    const bool do_f = a->f_host != nullptr;
    const bool do_y = a->v_host != nullptr && a->y_host != nullptr;
    const bool do_g = a->cot_host != nullptr && (a->g_u_host || a->g_udot_host || a->g_mu_lambda_host);
    if (!do_f && !do_y && !do_g) return fail(TLFE_E_INVALID, "tlfe_step_host: no operation requested");
    if (!m->host_stage) {
        tlfe_status st = make_stage(m);
        if (st != TLFE_OK) return st;
    }
    HostStage &h = *m->host_stage;
    cudaStream_t s = (cudaStream_t)stream;
    const int b = (int)(h.calls & 1);
    char *du = h.d_in[b], *dud = du + h.nu, *dv = dud + h.nb, *dcot = dv + h.nb;
    char *df = h.d_out[b], *dy = df + h.nb, *dgu = dy + h.nb, *dgud = dgu + h.nb, *dgth = dgud + h.nb;
    // inputs of set b, once the last computation that read them has ended
    if (h.used[b]) CKH(cudaStreamWaitEvent(h.h2d, h.comp_done[b], 0));
    CKH(cudaMemcpyAsync(du, a->u_host, h.nu, cudaMemcpyHostToDevice, h.h2d));
    if (a->udot_host) CKH(cudaMemcpyAsync(dud, a->udot_host, h.nb, cudaMemcpyHostToDevice, h.h2d));
    if (do_y) CKH(cudaMemcpyAsync(dv, a->v_host, h.nb, cudaMemcpyHostToDevice, h.h2d));
    if (do_g) CKH(cudaMemcpyAsync(dcot, a->cot_host, h.nb, cudaMemcpyHostToDevice, h.h2d));
    CKH(cudaEventRecord(h.in_ready[b], h.h2d));
    // the operations, once the inputs are in and set b's previous outputs are out
    CKH(cudaStreamWaitEvent(s, h.in_ready[b], 0));
    if (h.used[b]) CKH(cudaStreamWaitEvent(s, h.out_done[b], 0));
    const void *ud = a->udot_host ? dud : nullptr;
    tlfe_status st = TLFE_OK;
    if (do_f && do_y && fm_eligible(m)) {  // one fused pass for both
        st = check_force_matvec(m, du, dv, df, dy, a->a_M, a->a_K, a->a_C);
        if (st == TLFE_OK) st = force_matvec_op(m, du, ud, dv, a->a_M, a->a_K, a->a_C, df, dy, s);
        if (st != TLFE_OK) return st;
        CKH(cudaEventRecord(h.op_done[b][0], s));
        CKH(cudaEventRecord(h.op_done[b][1], s));
    } else {
    if (do_f) {
        st = tlfe_internal_force(m, du, ud, df, stream);
        if (st != TLFE_OK) return st;
        CKH(cudaEventRecord(h.op_done[b][0], s));
    }
    if (do_y) {
        st = tlfe_tangent_matvec(m, du, ud, dv, a->a_M, a->a_K, a->a_C, dy, stream);
        if (st != TLFE_OK) return st;
        CKH(cudaEventRecord(h.op_done[b][1], s));
    }
    }
    if (do_g) {
        st = tlfe_vjp(m, du, ud, dcot, a->g_u_host ? dgu : nullptr, a->g_udot_host ? dgud : nullptr,
                      a->g_mu_lambda_host ? (double *)dgth : nullptr, stream);
        if (st != TLFE_OK) return st;
        CKH(cudaEventRecord(h.op_done[b][2], s));
    }
    CKH(cudaEventRecord(h.comp_done[b], s));
    // outputs, each as soon as its operation has ended
    if (do_f) {
        CKH(cudaStreamWaitEvent(h.d2h, h.op_done[b][0], 0));
        CKH(cudaMemcpyAsync(a->f_host, df, h.nb, cudaMemcpyDeviceToHost, h.d2h));
    }
    if (do_y) {
        CKH(cudaStreamWaitEvent(h.d2h, h.op_done[b][1], 0));
        CKH(cudaMemcpyAsync(a->y_host, dy, h.nb, cudaMemcpyDeviceToHost, h.d2h));
    }
    if (do_g) {
        CKH(cudaStreamWaitEvent(h.d2h, h.op_done[b][2], 0));
        if (a->g_u_host) CKH(cudaMemcpyAsync(a->g_u_host, dgu, h.nb, cudaMemcpyDeviceToHost, h.d2h));
        if (a->g_udot_host) CKH(cudaMemcpyAsync(a->g_udot_host, dgud, h.nb, cudaMemcpyDeviceToHost, h.d2h));
        if (a->g_mu_lambda_host)
            CKH(cudaMemcpyAsync(a->g_mu_lambda_host, dgth, h.ng, cudaMemcpyDeviceToHost, h.d2h));
    }
    CKH(cudaEventRecord(h.out_done[b], h.d2h));
    h.used[b] = true;
    ++h.calls;
    return TLFE_OK;
}

extern "C" tlfe_status tlfe_step_host_wait(tlfe_mesh *m)
{
    TLFE_TRACE("tlfe_step_host_wait");
    if (!m) return fail(TLFE_E_INVALID, "mesh is NULL");
    if (!m->host_stage) return TLFE_OK;
    CKH(cudaStreamSynchronize(m->host_stage->h2d));
    CKH(cudaStreamSynchronize(m->host_stage->d2h));
    return TLFE_OK;
}
