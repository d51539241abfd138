// GMRES solve with FP64 iterative refinement (Section VI.C).
#include "vie_internal.cuh"

int solve_impl(const vie_op*, const void*, const void*, void*, int, int, int, const vie_solve_opts*,
               vie_solve_info*, cudaStream_t) {
  set_error("vie_solve is not available in this build");
  return VIE_ERR_ARG;
}

void solver_release(vie_op*) {}
