// bucket.cu -- hybrid column-bucket path (placeholder until implemented).
#include "common.cuh"
#include "internal.hpp"

namespace fsp {

bool bucket_supported(int64_t, int32_t, const KeyLayout &, const fsparse_config &) { return false; }

fsparse_status bucket_symbolic(const int32_t *, const int32_t *, const double *, double *, int64_t,
                               int32_t, int32_t, const KeyLayout &, const fsparse_config &, Plan &,
                               DevStatus *, Scratch &, cudaStream_t) {
    return set_error(FSPARSE_ERR_ARG, "bucket path unavailable");
}

}  // namespace fsp
