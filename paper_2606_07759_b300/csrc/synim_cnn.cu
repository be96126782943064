// synim_cnn.cu -- the learned misregistration estimator (BF16 CNN).
#include <string>

#include "synim_internal.h"

namespace synim {

cudaError_t cnn_predict_slopes(synim_ctx *c, const float *y, long long n, double *params_out, cudaStream_t st,
                               std::string &why) {
    (void)c; (void)y; (void)n; (void)params_out; (void)st;
    why = "the network has not been trained (synim_cnn_train) or loaded";
    return cudaErrorNotReady;
}

}  // namespace synim
