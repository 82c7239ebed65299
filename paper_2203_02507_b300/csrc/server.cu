// Serving: placeholder until the continuous-batching server lands.
#include "internal.h"
#include "runtime.h"


extern "C" {
int fpm_server_create(size_t, fpm_server **out) {
  if (out) *out = nullptr;
  return fpm::fail(FPM_ESTATE, "server not available in this build");
}
int fpm_submit(fpm_server *, fpm_plan *, int32_t, fpm_job *) { return fpm::fail(FPM_ESTATE, "server not available"); }
int fpm_poll(fpm_server *, fpm_job, int32_t *, double *, double *) { return fpm::fail(FPM_ESTATE, "server not available"); }
int fpm_server_destroy(fpm_server *) { return FPM_OK; }
}
