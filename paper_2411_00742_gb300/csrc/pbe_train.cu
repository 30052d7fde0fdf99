// Optimizer step for the learned closure: Adam (Kingma & Ba) on device
// arrays, the update the paper's parameter estimation uses (Appendix C).
#include <cmath>

#include "pbe_internal.h"

void pbe_set_error_message(int code, const char* msg);  // pbe_api.cu

namespace {

__global__ void k_adam(double* w, const double* grad, double* m, double* v, int n, double lr, double b1, double b2,
                       double eps, double c1, double c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double gi = grad[i];
        const double mi = b1 * m[i] + (1.0 - b1) * gi;
        const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
    }
}

}  // namespace

extern "C" pbe_status pbe_adam_update(double* w, const double* grad, double* m, double* v, int n, double lr,
                                      double beta1, double beta2, double eps, int step, void* stream)
{
    if (!w || !grad || !m || !v || n < 1 || step < 1) {
        pbe_set_error_message(PBE_EINVAL, "pbe_adam_update: invalid argument");
        return PBE_EINVAL;
    }
    if (!(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0)) {
        pbe_set_error_message(PBE_EINVAL, "pbe_adam_update: invalid hyper-parameters");
        return PBE_EINVAL;
    }
    const double c1 = 1.0 - std::pow(beta1, step), c2 = 1.0 - std::pow(beta2, step);
    const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    k_adam<<<blocks, 256, 0, (cudaStream_t)stream>>>(w, grad, m, v, n, lr, beta1, beta2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        pbe_set_error_message(PBE_ECUDA, cudaGetErrorString(e));
        return PBE_ECUDA;
    }
    return PBE_OK;
}
