// k_loop.cu -- the pseudo-transient continuation of one implicit stage
// (Section 2.4) as a device-side loop: a CUDA graph whose WHILE node repeats
// {controller; IF refresh: V-cycle with smoother rebuild; IF plain: V-cycle}
// until the controller clears the loop condition.  The host then synchronises
// once per stage instead of once per V-cycle.
//
// The controller is one thread.  At the start of pseudo-iteration m it reads
// ||F^m||^2 (left by the previous V-cycle's final residual, or by the stage's
// first residual evaluation) and applies, in this order, the same rules as
// the host loop of api.cu:
//   1. a singular block flagged by the last rebuild, or a bulk-copy wait
//      that gave up, ends the stage with that error;
//   2. ||F^m|| <= tol ||F^0|| (or ||F^0|| = 0) ends it converged;
//   3. a non-finite norm ends it with PMG_ENONFINITE;
//   4. m >= max_pseudo ends it with PMG_ENOTCONV;
//   5. otherwise dtau follows SER (eq. ser, exponent 1.5, capped at
//      dtau_max), the smoother is rebuilt at m = 0 and every refresh_every
//      iterations until one rebuild used dtau_max (or always), and one of the
//      two V-cycle branches is enabled.
// Whatever the state it reads, the controller stops the loop once its own
// iteration count passes max_pseudo + 2, so the WHILE node always ends.
#include "pmg_internal.h"

namespace pmg {

__global__ void stage_loop_controller(LoopState* st, const double* __restrict__ scal, int* sing_flag,
                                      double* __restrict__ d_dtau, double* __restrict__ hist_norm,
                                      double* __restrict__ hist_dtau, LoopParams prm,
                                      cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_refresh,
                                      cudaGraphConditionalHandle h_plain) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = st->m;
  const double nm = sqrt(scal[0]);
  int status = LOOP_RUNNING;
  if (m > prm.max_pseudo + 2) status = LOOP_NOTCONV;   // hard bound on the number of bodies
  else if (*sing_flag) status = LOOP_SINGULAR;
  else if (scal[1] != 0.0) status = LOOP_TIMEOUT;
  if (status == LOOP_RUNNING) {
    if (m == 0) st->n0 = nm;
    const double n0 = st->n0;
    const double next_dtau = m > 0 ? fmin(st->dtau * pow(st->prev / nm, 1.5), st->dtau_max) : st->dtau;
    if (m <= prm.max_pseudo) {
      hist_norm[m] = nm;
      hist_dtau[m] = next_dtau;
    }
    if (nm <= prm.tol * n0 || n0 == 0.0) status = LOOP_CONVERGED;
    else if (!isfinite(nm)) status = LOOP_NONFINITE;
    else if (m >= prm.max_pseudo) status = LOOP_NOTCONV;
    if (status == LOOP_RUNNING) {
      st->dtau = next_dtau;
      const bool refresh =
          (m == 0) || (m % prm.refresh_every == 0 && (prm.refresh_always || st->built < st->dtau_max));
      if (refresh) {
        st->built = st->dtau;
        *d_dtau = st->dtau;
        st->n_refresh += 1;
      }
      st->prev = nm;
      st->m = m + 1;
      cudaGraphSetConditional(h_refresh, refresh ? 1u : 0u);
      cudaGraphSetConditional(h_plain, refresh ? 0u : 1u);
      return;
    }
  }
  // the stage ends here: no V-cycle in this body, and no further body
  st->status = status;
  st->final_norm = nm;
  st->iters = m;
  cudaGraphSetConditional(h_refresh, 0u);
  cudaGraphSetConditional(h_plain, 0u);
  cudaGraphSetConditional(h_loop, 0u);
}

void launch_loop_controller(LoopState* st, const double* scal, int* sing_flag, double* d_dtau, double* hist_norm,
                            double* hist_dtau, const LoopParams& prm, cudaGraphConditionalHandle h_loop,
                            cudaGraphConditionalHandle h_refresh, cudaGraphConditionalHandle h_plain,
                            cudaStream_t s) {
  stage_loop_controller<<<1, 32, 0, s>>>(st, scal, sing_flag, d_dtau, hist_norm, hist_dtau, prm, h_loop,
                                          h_refresh, h_plain);
}

}  // namespace pmg
