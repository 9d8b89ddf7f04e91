// Split-precision tensor-core path (placeholder until the tcgen05 kernels land).
#include "exx_internal.h"

namespace exx {

static int unsupported(const char *what)
{
    set_error(std::string(what) + ": split-precision path not built yet");
    return EXX_ERR_UNSUPPORTED;
}

int tc_upload(Plan &, int) { return unsupported("tc_upload"); }
int tc_prepare_orbitals(Plan &, const double *, int, long, const double *, const double *, int, long, bool,
                        cudaStream_t)
{
    return unsupported("tc_prepare_orbitals");
}
int tc_solve_batch(Plan &, int, const int2 *, int, float *, float *, cudaStream_t) { return unsupported("tc_solve_batch"); }
int tc_accumulate(Plan &, const Block *, int, const float *, cudaStream_t) { return unsupported("tc_accumulate"); }
int tc_finalize(Plan &, int, double *, long, cudaStream_t) { return unsupported("tc_finalize"); }

}  // namespace exx
