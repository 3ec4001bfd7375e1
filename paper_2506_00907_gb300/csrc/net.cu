// net.cu -- the warm-start network: a 4-layer perceptron (4 -> 64 -> 64 -> 64
// -> 2, tanh hidden layers, linear output) trained on the GPU by this file's
// own forward, backward and Adam kernels, and the kernel that turns its
// prediction into the initial fields of a pipe case.  The paper has no
// network; it only supplies the steady fields a warm start approaches.
//
// Precision: FP32 master parameters and Adam moments; the forward and
// backward passes read an FP16 copy of the weights and accumulate in FP32.
// Parameter layout (one flat vector, layer by layer): W_l (rows = outputs,
// row-major) then b_l.
#include <cuda_fp16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "lbm.h"

namespace lbm_net_impl {

constexpr int D0 = 4, H = 64, DL = 2;
constexpr int NL = 4;                                      // layers
// layer widths {4, 64, 64, 64, 2}
__host__ __device__ constexpr int dim_of(int l) { return l == 0 ? D0 : (l == NL ? DL : H); }
constexpr int NPARAM = H * D0 + H + H * H + H + H * H + H + DL * H + DL;
constexpr int CHUNK = 64;                                  // samples per block iteration = threads per block
constexpr int PAD = H + 1;                                 // padded row of an activation / delta tile

__host__ __device__ constexpr int w_off(int l) {           // offset of W_l (l = 0..3)
    return l == 0 ? 0 : w_off(l - 1) + dim_of(l) * dim_of(l - 1) + dim_of(l);
}
__host__ __device__ constexpr int b_off(int l) { return w_off(l) + dim_of(l + 1) * dim_of(l); }

struct Smem {
    __half w[NPARAM];                 // FP16 weights (all layers)
    float act[4][CHUNK][PAD];         // a_0 (x) .. a_3 per sample, padded rows
    float dlt[CHUNK][PAD];            // delta of the layer being back-propagated
    float grad[NPARAM];               // this block's gradient
    double loss[CHUNK];
};

__device__ __forceinline__ float wv(const Smem &s, int l, int o, int i) {
    return __half2float(s.w[w_off(l) + o * dim_of(l) + i]);
}
__device__ __forceinline__ float bv(const Smem &s, int l, int o) { return __half2float(s.w[b_off(l) + o]); }

// forward of sample `t` of the chunk; act[0][t] holds x; returns y
__device__ void forward_chunk(Smem &s, int t, float y[DL]) {
    for (int l = 0; l < NL; ++l) {
        const int in = dim_of(l), out = dim_of(l + 1);
        float a[H];
#pragma unroll
        for (int i = 0; i < H; ++i) a[i] = i < in ? s.act[l][t][i] : 0.f;
        for (int o = 0; o < out; ++o) {
            float z = bv(s, l, o);
#pragma unroll
            for (int i = 0; i < H; ++i)
                if (i < in) z = fmaf(wv(s, l, o, i), a[i], z);
            if (l < NL - 1) s.act[l + 1][t][o] = tanhf(z);
            else y[o] = z;
        }
    }
}

__global__ void __launch_bounds__(CHUNK) k_net_forward(const __half *w, const float *x, float *y, int64_t n) {
    extern __shared__ __align__(16) unsigned char raw[];
    Smem &s = *reinterpret_cast<Smem *>(raw);
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) s.w[i] = w[i];
    __syncthreads();
    const int t = threadIdx.x;
    for (int64_t base = (int64_t)blockIdx.x * CHUNK; base < n; base += (int64_t)gridDim.x * CHUNK) {
        const int64_t i = base + t;
        if (i < n) {
            for (int k = 0; k < D0; ++k) s.act[0][t][k] = x[i * D0 + k];
            float out[DL];
            forward_chunk(s, t, out);
            for (int k = 0; k < DL; ++k) y[i * DL + k] = out[k];
        }
    }
}

// Loss (mean squared error over n samples and DL outputs) and its gradient,
// accumulated into grad (FP32) and loss (FP64).
__global__ void __launch_bounds__(CHUNK) k_net_grad(const __half *w, const float *x, const float *target, int64_t n,
                                                    float *grad, double *loss) {
    extern __shared__ __align__(16) unsigned char raw[];
    Smem &s = *reinterpret_cast<Smem *>(raw);
    const int t = threadIdx.x;
    for (int i = t; i < NPARAM; i += blockDim.x) {
        s.w[i] = w[i];
        s.grad[i] = 0.f;
    }
    s.loss[t] = 0.0;
    const float scale = 2.0f / (float)((double)n * DL);
    __syncthreads();
    for (int64_t base = (int64_t)blockIdx.x * CHUNK; base < n; base += (int64_t)gridDim.x * CHUNK) {
        const int64_t i = base + t;
        const bool live = i < n;
        // ---- forward
        float y[DL] = {0.f, 0.f}, d_out[DL] = {0.f, 0.f};
        for (int k = 0; k < D0; ++k) s.act[0][t][k] = live ? x[i * D0 + k] : 0.f;
        forward_chunk(s, t, y);
        if (live) {
            for (int k = 0; k < DL; ++k) {
                const float e = y[k] - target[i * DL + k];
                s.loss[t] += (double)e * e;
                d_out[k] = scale * e;                  // dL/dy
            }
        }
        // ---- backward, layer by layer (dead samples carry zero deltas)
        for (int k = 0; k < DL; ++k) s.dlt[t][k] = d_out[k];
        __syncthreads();
        for (int l = NL - 1; l >= 0; --l) {
            const int in = dim_of(l), out = dim_of(l + 1);
            // gradient rows owned by thread o: dW_l[o][j] += sum_s dlt[s][o] act_l[s][j], db_l[o] += sum_s dlt[s][o]
            for (int o = t; o < out; o += blockDim.x) {
                float gb = 0.f;
                for (int smp = 0; smp < CHUNK; ++smp) gb += s.dlt[smp][o];
                s.grad[b_off(l) + o] += gb;
                for (int j = 0; j < in; ++j) {
                    float g = 0.f;
                    for (int smp = 0; smp < CHUNK; ++smp) g = fmaf(s.dlt[smp][o], s.act[l][smp][j], g);
                    s.grad[w_off(l) + o * in + j] += g;
                }
            }
            if (l == 0) break;
            // delta of the layer below: (W_l^T dlt) * (1 - a_l^2)
            float dn[H];
#pragma unroll
            for (int j = 0; j < H; ++j) dn[j] = 0.f;
            for (int o = 0; o < out; ++o) {
                const float d = s.dlt[t][o];
#pragma unroll
                for (int j = 0; j < H; ++j)
                    if (j < in) dn[j] = fmaf(wv(s, l, o, j), d, dn[j]);
            }
            __syncthreads();                           // every thread is done reading dlt
#pragma unroll
            for (int j = 0; j < H; ++j)
                if (j < in) {
                    const float a = s.act[l][t][j];
                    s.dlt[t][j] = dn[j] * (1.f - a * a);
                }
            __syncthreads();
        }
        __syncthreads();
    }
    __syncthreads();
    for (int k = t; k < NPARAM; k += blockDim.x) atomicAdd(&grad[k], s.grad[k]);
    // block loss in a fixed order
    if (t == 0) {
        double tot = 0.0;
        for (int k = 0; k < CHUNK; ++k) tot += s.loss[k];
        atomicAdd(loss, tot);
    }
}

// Adam with bias correction; writes the FP16 copy and clears the gradient.
__global__ void k_net_adam(float *p, float *m, float *v, float *g, __half *w16, int np, float lr, float b1, float b2,
                           float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    w16[i] = __float2half_rn(pi);
    g[i] = 0.f;
}

__global__ void k_to_half(const float *p, __half *w16, int np) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) w16[i] = __float2half_rn(p[i]);
}

// Initial fields of a pipe case from the network: features (x2/R, x3/R,
// f_Ha, f_cw) per fluid node, prediction (u_hat, b_hat), u_x = u_hat * us,
// B = (b_hat * bs, B0, 0); solid nodes get rest values.
__global__ void __launch_bounds__(CHUNK) k_net_pipe_fields(const __half *w, int nx, int ny, int nz, float R, float fHa,
                                                           float fcw, float us, float bs, float B0, float *u, float *B) {
    extern __shared__ __align__(16) unsigned char raw[];
    Smem &s = *reinterpret_cast<Smem *>(raw);
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) s.w[i] = w[i];
    __syncthreads();
    const int t = threadIdx.x;
    const int64_t N = (int64_t)nx * ny * nz;
    const float cy = 0.5f * (ny - 1), cz = 0.5f * (nz - 1);
    for (int64_t base = (int64_t)blockIdx.x * CHUNK; base < N; base += (int64_t)gridDim.x * CHUNK) {
        const int64_t n = base + t;
        if (n >= N) continue;
        const int y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
        const float ry = (y - cy) / R, rz = (z - cz) / R;
        s.act[0][t][0] = ry;
        s.act[0][t][1] = rz;
        s.act[0][t][2] = fHa;
        s.act[0][t][3] = fcw;
        float out[DL];
        forward_chunk(s, t, out);
        const bool fluid = ry * ry + rz * rz < 1.f;
        u[3 * n + 0] = fluid ? out[0] * us : 0.f;
        u[3 * n + 1] = 0.f;
        u[3 * n + 2] = 0.f;
        B[3 * n + 0] = fluid ? out[1] * bs : 0.f;
        B[3 * n + 1] = B0;
        B[3 * n + 2] = 0.f;
    }
}

}  // namespace lbm_net_impl

using namespace lbm_net_impl;

struct lbm_net {
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    __half *w16 = nullptr;
    double *loss = nullptr;
    int64_t steps = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 1;
};

namespace {
size_t smem_bytes() { return sizeof(Smem); }
bool setup_attrs() {
    static bool done = false;
    if (done) return true;
    const int b = (int)smem_bytes();
    if (cudaFuncSetAttribute(k_net_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, b) != cudaSuccess) return false;
    if (cudaFuncSetAttribute(k_net_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, b) != cudaSuccess) return false;
    if (cudaFuncSetAttribute(k_net_pipe_fields, cudaFuncAttributeMaxDynamicSharedMemorySize, b) != cudaSuccess) return false;
    done = true;
    return true;
}
int grid_for(const lbm_net *net, int64_t n) {
    const int64_t blocks = (n + CHUNK - 1) / CHUNK;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, 2 * net->sm_count));
}
}  // namespace

extern "C" {

int64_t lbm_net_num_params(void) { return NPARAM; }

lbm_status lbm_net_create(const int32_t *dims, int32_t ndims, const float *init, void *stream, lbm_net **out) {
    if (!out || !dims || !init || ndims != NL + 1) return LBM_EINVAL;
    *out = nullptr;
    for (int i = 0; i <= NL; ++i)
        if (dims[i] != dim_of(i)) return LBM_EINVAL;
    if (!setup_attrs()) return LBM_ECUDA;
    lbm_net *net = new lbm_net();
    net->stream = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&net->sm_count, cudaDevAttrMultiProcessorCount, dev);
    const size_t fb = NPARAM * sizeof(float);
    bool ok = cudaMalloc(&net->p, fb) == cudaSuccess && cudaMalloc(&net->m, fb) == cudaSuccess &&
              cudaMalloc(&net->v, fb) == cudaSuccess && cudaMalloc(&net->g, fb) == cudaSuccess &&
              cudaMalloc(&net->w16, NPARAM * sizeof(__half)) == cudaSuccess &&
              cudaMalloc(&net->loss, sizeof(double)) == cudaSuccess;
    ok = ok && cudaMemcpy(net->p, init, fb, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(net->m, 0, fb) == cudaSuccess && cudaMemset(net->v, 0, fb) == cudaSuccess &&
         cudaMemset(net->g, 0, fb) == cudaSuccess;
    if (ok) {
        k_to_half<<<(NPARAM + 255) / 256, 256, 0, net->stream>>>(net->p, net->w16, NPARAM);
        ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(net->stream) == cudaSuccess;
    }
    if (!ok) {
        lbm_net_destroy(net);
        return LBM_ENOMEM;
    }
    *out = net;
    return LBM_OK;
}

void lbm_net_destroy(lbm_net *net) {
    if (!net) return;
    cudaFree(net->p);
    cudaFree(net->m);
    cudaFree(net->v);
    cudaFree(net->g);
    cudaFree(net->w16);
    cudaFree(net->loss);
    delete net;
}

lbm_status lbm_net_get_params(lbm_net *net, float *host) {
    if (!net || !host) return LBM_EINVAL;
    if (cudaMemcpy(host, net->p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ECUDA;
    return LBM_OK;
}

lbm_status lbm_net_set_params(lbm_net *net, const float *host) {
    if (!net || !host) return LBM_EINVAL;
    if (cudaMemcpy(net->p, host, NPARAM * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return LBM_ECUDA;
    k_to_half<<<(NPARAM + 255) / 256, 256, 0, net->stream>>>(net->p, net->w16, NPARAM);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(net->stream) != cudaSuccess) return LBM_ECUDA;
    net->steps = 0;
    cudaMemset(net->m, 0, NPARAM * sizeof(float));
    cudaMemset(net->v, 0, NPARAM * sizeof(float));
    return LBM_OK;
}

lbm_status lbm_net_forward(lbm_net *net, const float *x, float *y, int64_t n) {
    if (!net || !x || !y || n < 0) return LBM_EINVAL;
    if (n == 0) return LBM_OK;
    k_net_forward<<<grid_for(net, n), CHUNK, smem_bytes(), net->stream>>>(net->w16, x, y, n);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

lbm_status lbm_net_loss_grad(lbm_net *net, const float *x, const float *t, int64_t n, double *loss, float *grad) {
    if (!net || !x || !t || n < 1) return LBM_EINVAL;
    if (cudaMemsetAsync(net->loss, 0, sizeof(double), net->stream) != cudaSuccess) return LBM_ECUDA;
    k_net_grad<<<grid_for(net, n), CHUNK, smem_bytes(), net->stream>>>(net->w16, x, t, n, net->g, net->loss);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    if (loss) {
        double tot = 0;
        if (cudaMemcpyAsync(&tot, net->loss, sizeof(double), cudaMemcpyDeviceToHost, net->stream) != cudaSuccess)
            return LBM_ECUDA;
        if (cudaStreamSynchronize(net->stream) != cudaSuccess) return LBM_ECUDA;
        *loss = tot / ((double)n * DL);
    }
    if (grad) {
        if (cudaMemcpyAsync(grad, net->g, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, net->stream) != cudaSuccess)
            return LBM_ECUDA;
        if (cudaStreamSynchronize(net->stream) != cudaSuccess) return LBM_ECUDA;
    }
    return LBM_OK;
}

lbm_status lbm_net_adam(lbm_net *net, float lr, float beta1, float beta2, float eps) {
    if (!net) return LBM_EINVAL;
    net->steps += 1;
    const float c1 = 1.f - std::pow(beta1, (float)net->steps), c2 = 1.f - std::pow(beta2, (float)net->steps);
    k_net_adam<<<(NPARAM + 255) / 256, 256, 0, net->stream>>>(net->p, net->m, net->v, net->g, net->w16, NPARAM, lr,
                                                              beta1, beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

lbm_status lbm_net_pipe_fields(lbm_net *net, int32_t nx, int32_t ny, int32_t nz, double R, double f_ha, double f_cw,
                               double u_scale, double b_scale, double B0, float *u, float *B) {
    if (!net || !u || !B || nx < 1 || ny < 1 || nz < 1 || !(R > 0)) return LBM_EINVAL;
    const int64_t N = (int64_t)nx * ny * nz;
    k_net_pipe_fields<<<grid_for(net, N), CHUNK, smem_bytes(), net->stream>>>(
        net->w16, nx, ny, nz, (float)R, (float)f_ha, (float)f_cw, (float)u_scale, (float)b_scale, (float)B0, u, B);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

}  // extern "C"
