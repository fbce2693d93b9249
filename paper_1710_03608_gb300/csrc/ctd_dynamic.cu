// CTD-D (Algorithm 2): placeholder until the dynamic path lands.
#include "ctd_internal.cuh"

using namespace ctd;

struct ctd_factors::Dyn {};

extern "C" ctd_status ctd_dynamic_create(const int64_t dims2[2], int alpha, int precision,
                                         uint64_t seed, uint64_t stream_id, ctd_factors** state) {
  (void)dims2; (void)alpha; (void)precision; (void)seed; (void)stream_id; (void)state;
  return fail(CTD_ENOTSUP, "CTD-D is not built yet");
}

extern "C" ctd_status ctd_dynamic_step(ctd_factors* state, const ctd_coo3* dX, int64_t d,
                                       double eps, void* stream) {
  (void)state; (void)dX; (void)d; (void)eps; (void)stream;
  return fail(CTD_ENOTSUP, "CTD-D is not built yet");
}

extern "C" ctd_status ctd_get_step(const ctd_factors* F, int64_t t, int64_t info[4], double sq[2]) {
  (void)F; (void)t; (void)info; (void)sq;
  return fail(CTD_ENOTSUP, "CTD-D is not built yet");
}

extern "C" ctd_status ctd_get_M(const ctd_factors* F, int64_t t, double* M) {
  (void)F; (void)t; (void)M;
  return fail(CTD_ENOTSUP, "CTD-D is not built yet");
}
