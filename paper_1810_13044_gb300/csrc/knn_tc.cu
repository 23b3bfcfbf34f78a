// bfloat16 tensor-core (tcgen05) candidate tiles for the kNN graph.
#include <cuda_bf16.h>

#include "slk_internal.cuh"

slk_status knn_cand_bf16_launch(slk_ctx* ctx, const __nv_bfloat16*, const float*, int64_t, int,
                                int64_t, int, int, float*, int32_t*) {
    return set_err(ctx, SLK_ERR_INVALID_ARG, "SLK_KNN_BF16_RERANK is not available in this build");
}
