// Backward-Euler Newton/CG step (Section 7 without constraints).
#include "tlfe_mesh.h"

namespace tlfe {
struct NewtonState {};
void destroy_newton(tlfe_mesh *m)
{
    delete m->newton;
    m->newton = nullptr;
}
}  // namespace tlfe

extern "C" tlfe_status tlfe_newton_step(tlfe_mesh *m, const double *, const double *, const tlfe_step_params *,
                                        double *, tlfe_step_report *, void *)
{
    if (!m) return tlfe::fail(TLFE_E_INVALID, "mesh is NULL");
    return tlfe::fail(TLFE_E_UNSUPPORTED, "newton step not built yet");
}
