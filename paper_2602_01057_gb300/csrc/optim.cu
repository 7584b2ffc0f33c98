// Parameter chain (a6), loss and residual (a4), Adam (a7).
#include "rgrt_internal.h"

namespace rgrt {
namespace {

// dL/d(P, S) accumulated per Gaussian -> dL/d(log-scale, quaternion).
//   P = R diag(e^{-2 l}) R^T,  S = Sigma/det Sigma = R diag(e^{-2(l_b + l_c)}) R^T
//   dL/dl_k = -2 e^{-2 l_k} r_k^T G_P r_k - 2 sum_{j != k} e^{-2(l_a + l_b)}_j r_j^T G_S r_j
//   dL/dR   = 2 G_P R D_P + 2 G_S R D_S
// then through R(w, x, y, z) of the normalised quaternion and the
// normalisation q / |q|.
__global__ void k_param_chain(const float *__restrict__ mu, const float *__restrict__ ls,
                              const float *__restrict__ q, const float *__restrict__ rho,
                              int64_t n, const float4 *__restrict__ grad, float *g_mu, float *g_ls,
                              float *g_q, float *g_rho)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float4 a = grad[GRAD_F4 * k], b = grad[GRAD_F4 * k + 1], c = grad[GRAD_F4 * k + 2],
           d = grad[GRAD_F4 * k + 3];
    if (g_mu) { g_mu[3 * k] = a.x; g_mu[3 * k + 1] = a.y; g_mu[3 * k + 2] = a.z; }
    if (g_rho) g_rho[k] = a.w;
    if (!g_ls && !g_q) return;
    float GP[3][3] = { { b.x, b.y, b.z }, { b.y, b.w, c.x }, { b.z, c.x, c.y } };
    float GS[3][3] = { { c.z, c.w, d.x }, { c.w, d.y, d.z }, { d.x, d.z, d.w } };
    float qw = q[4 * k], qx = q[4 * k + 1], qy = q[4 * k + 2], qz = q[4 * k + 3];
    float nq = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    float w, x, y, z;
    if (!(nq > 0.0f)) { w = 1.0f; x = y = z = 0.0f; nq = 1.0f; }
    else { float inv = 1.0f / nq; w = qw * inv; x = qx * inv; y = qy * inv; z = qz * inv; }
    float R[3][3] = {
        { 1.0f - 2.0f * (y * y + z * z), 2.0f * (x * y - w * z), 2.0f * (x * z + w * y) },
        { 2.0f * (x * y + w * z), 1.0f - 2.0f * (x * x + z * z), 2.0f * (y * z - w * x) },
        { 2.0f * (x * z - w * y), 2.0f * (y * z + w * x), 1.0f - 2.0f * (x * x + y * y) } };
    float l[3] = { ls[3 * k], ls[3 * k + 1], ls[3 * k + 2] };
    float DP[3] = { expf(-2.0f * l[0]), expf(-2.0f * l[1]), expf(-2.0f * l[2]) };
    float DS[3] = { expf(-2.0f * (l[1] + l[2])), expf(-2.0f * (l[0] + l[2])), expf(-2.0f * (l[0] + l[1])) };
    // column projections r_k^T G r_k and G R
    float GPR[3][3], GSR[3][3], qp[3], qs[3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            GPR[i][j] = GP[i][0] * R[0][j] + GP[i][1] * R[1][j] + GP[i][2] * R[2][j];
            GSR[i][j] = GS[i][0] * R[0][j] + GS[i][1] * R[1][j] + GS[i][2] * R[2][j];
        }
#pragma unroll
    for (int j = 0; j < 3; j++) {
        qp[j] = R[0][j] * GPR[0][j] + R[1][j] * GPR[1][j] + R[2][j] * GPR[2][j];
        qs[j] = R[0][j] * GSR[0][j] + R[1][j] * GSR[1][j] + R[2][j] * GSR[2][j];
    }
    if (g_ls) {
        g_ls[3 * k + 0] = -2.0f * (DP[0] * qp[0] + DS[1] * qs[1] + DS[2] * qs[2]);
        g_ls[3 * k + 1] = -2.0f * (DP[1] * qp[1] + DS[0] * qs[0] + DS[2] * qs[2]);
        g_ls[3 * k + 2] = -2.0f * (DP[2] * qp[2] + DS[0] * qs[0] + DS[1] * qs[1]);
    }
    if (!g_q) return;
    float Gr[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) Gr[i][j] = 2.0f * (GPR[i][j] * DP[j] + GSR[i][j] * DS[j]);
    float gw = 2.0f * (z * (Gr[1][0] - Gr[0][1]) + y * (Gr[0][2] - Gr[2][0]) + x * (Gr[2][1] - Gr[1][2]));
    float gx = 2.0f * (y * (Gr[0][1] + Gr[1][0]) + z * (Gr[0][2] + Gr[2][0]) + w * (Gr[2][1] - Gr[1][2]))
               - 4.0f * x * (Gr[1][1] + Gr[2][2]);
    float gy = 2.0f * (x * (Gr[0][1] + Gr[1][0]) + z * (Gr[1][2] + Gr[2][1]) + w * (Gr[0][2] - Gr[2][0]))
               - 4.0f * y * (Gr[0][0] + Gr[2][2]);
    float gz = 2.0f * (x * (Gr[0][2] + Gr[2][0]) + y * (Gr[1][2] + Gr[2][1]) + w * (Gr[1][0] - Gr[0][1]))
               - 4.0f * z * (Gr[0][0] + Gr[1][1]);
    float dot = gw * w + gx * x + gy * y + gz * z;
    float inv = 1.0f / nq;
    g_q[4 * k + 0] = (gw - w * dot) * inv;
    g_q[4 * k + 1] = (gx - x * dot) * inv;
    g_q[4 * k + 2] = (gy - y * dot) * inv;
    g_q[4 * k + 3] = (gz - z * dot) * inv;
    (void)mu; (void)rho;
}

constexpr int LOSS_BS = 256;
constexpr int LOSS_MAXBLK = 2048;

// mult / add (optional, per ray): the measurement model's multiplicative
// factor (attenuation, detector efficiency) and additive background (scatter,
// randoms): L2 compares mult I + add with y, Poisson takes the mean
// kappa mult I + add + eps.
__global__ void k_loss(int kind, const float *__restrict__ I, const float *__restrict__ y, int64_t n,
                       float kappa, float eps, const float *__restrict__ mult,
                       const float *__restrict__ add, float *__restrict__ dLdI, double *partial)
{
    __shared__ double sh[LOSS_BS / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float Ii = I[i], yi = y[i];
        const float mi = mult ? mult[i] : 1.0f;
        const float mI = mult ? mi * Ii : Ii;
        if (kind == 0) {
            float r = mI - yi;
            if (add) r += add[i];
            s += 0.5 * (double)r * (double)r;
            dLdI[i] = mult ? mi * r : r;
        } else {
            float lam = kappa * mI + eps;
            if (add) lam += add[i];
            // the logarithm in binary32 (FP64 throughput is a small fraction
            // of FP32 on this GPU), the terms summed in binary64
            s += (double)lam - (double)yi * (double)logf(lam);
            dLdI[i] = mult ? kappa * mi * (1.0f - yi / lam) : kappa * (1.0f - yi / lam);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < LOSS_BS / 32; k++) t += sh[k];
        partial[blockIdx.x] = t;
    }
}

// acc (nullable): running total over several launches (ray ranges of one
// step).  One CTA of LOSS_BS threads, a fixed summation order (strided
// partial sums, then a tree), so the total does not vary from run to run.
__global__ void k_loss_final(const double *partial, int nblk, double *acc, float *loss_out)
{
    __shared__ double sh[LOSS_BS / 32];
    double t = 0.0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) t += partial[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < LOSS_BS / 32; k++) u += sh[k];
        if (acc) {
            u += *acc;
            *acc = u;
        }
        *loss_out = (float)u;
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2, const float *bc_dev, const uint32_t *skip)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (skip && *skip) return;
    if (bc_dev) { bc1 = bc_dev[0]; bc2 = bc_dev[1]; }
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float denom = sqrtf(vi / bc2) + eps;
    p[i] -= (lr / bc1) * mi / denom;
}

}  // namespace

cudaError_t launch_param_chain(const float *mu, const float *ls, const float *q, const float *rho,
                               int64_t n, const float4 *grad, float *g_mu, float *g_ls,
                               float *g_q, float *g_rho, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_param_chain<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mu, ls, q, rho, n, grad, g_mu, g_ls,
                                                               g_q, g_rho);
    count_launches(1);
    return cudaGetLastError();
}

int loss_blocks(int64_t n)
{
    int64_t b = (n + LOSS_BS - 1) / LOSS_BS;
    if (b > LOSS_MAXBLK) b = LOSS_MAXBLK;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_loss(int kind, const float *I, const float *y, int64_t n, float kappa,
                        float eps, const float *mult, const float *add, float *dLdI, double *partial,
                        int nblk, float *loss_out, cudaStream_t s, double *acc)
{
    k_loss<<<nblk, LOSS_BS, 0, s>>>(kind, I, y, n, kappa, eps, mult, add, dLdI, partial);
    k_loss_final<<<1, LOSS_BS, 0, s>>>(partial, nblk, acc, loss_out);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr,
                        float beta1, float beta2, float eps, float bc1, float bc2,
                        const float *bc_dev, const uint32_t *skip, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, g, m, v, n, lr, beta1, beta2, eps, bc1, bc2,
                                                       bc_dev, skip);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rgrt
