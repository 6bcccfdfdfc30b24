// ap_adjoint.cu -- discrete adjoint of the gather + push (row a13).
#include <cuda_runtime.h>

#include "ap_internal.h"

extern "C" {

size_t ap_adjoint_workspace_bytes(ap_handle h, int64_t n, int64_t n_steps, int32_t ckpt_every) {
  (void)h; (void)n; (void)n_steps; (void)ckpt_every;
  return 0;
}

int ap_push_adjoint(ap_handle h, const ap_particles *p0, const ap_grid *g, double t0, double dt,
                    int64_t n_steps, int32_t ckpt_every, int32_t objective, int32_t precision,
                    double *dJ_dparams, double *J_out, void *workspace, size_t ws_bytes,
                    void *stream) {
  (void)h; (void)p0; (void)g; (void)t0; (void)dt; (void)n_steps; (void)ckpt_every;
  (void)objective; (void)precision; (void)dJ_dparams; (void)J_out; (void)workspace;
  (void)ws_bytes; (void)stream;
  return AP_ERR_UNSUPPORTED;
}

}  // extern "C"
