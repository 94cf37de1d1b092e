// ensf_tc.cu -- tcgen05 tensor-core stages (placeholder until the kernels land).
#include "ensf_tc.h"

namespace ensf {

struct TcContext { int unused; };

cudaError_t tc_context_create(TcContext **out) { *out = nullptr; return cudaErrorNotSupported; }
void tc_context_destroy(TcContext *ctx) { delete ctx; }
int64_t tc_partial_floats(int max_n, int sms) { return 0; }
cudaError_t launch_gram_tc(TcContext *, const TcGramArgs &, int, int *, int64_t *, int *, cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_wx_em_tc(TcContext *, const TcWxArgs &, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace ensf
