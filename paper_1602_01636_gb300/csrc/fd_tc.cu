// Placeholder for the tensor-core (tcgen05) mixed-precision FD; replaced by
// the real implementation. Returns IGAFD_ERR_ARG so no caller silently gets a
// different precision.
#include "common.cuh"

igafd_status igafd_fd_tc_init(igafd_patch *, cudaStream_t) { return IGAFD_OK; }
void igafd_fd_tc_free(igafd_patch *) {}
igafd_status igafd_fd_tc_apply(igafd_patch *, igafd_dtype, const double *, double *, cudaStream_t,
                               double *) {
  return IGAFD_ERR_ARG;
}
