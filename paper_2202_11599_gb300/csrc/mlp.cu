// Learned warm start: a small multilayer perceptron (input -> hidden -> hidden ->
// output, erf-GELU hidden units) with BF16 weights used by forward and backward
// (FP32 accumulation), FP32 master weights, and an Adam optimiser.  The model maps
// the features of an x-subproblem (its right-hand side projected on the Nystrom
// basis U, rho, the ADMM iteration, log ||r||) to coefficients c so that the PCG
// starts at x_prev + U c instead of x_prev.  PCG still runs to the same tolerance.
//
// Parameter layout (FP32 master and BF16 copy): [W1 (h x i), b1 (h), W2 (h x h), b2 (h),
// W3 (o x h), b3 (o)], weights row-major (output x input).  Batches are row-major
// (B x features).  All reductions are in a fixed order (deterministic).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "device_util.cuh"
#include "solver.cuh"

using namespace nys;

struct nys_mlp_s {
  int n_in = 0, n_hid = 0, n_out = 0;
  int64_t n_params = 0;
  float* w32 = nullptr;          // master parameters
  __nv_bfloat16* w16 = nullptr;  // BF16 copy of the parameters used in matmuls
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  int step = 0;
  // activations for a batch (grown on demand)
  int cap = 0;
  float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *y = nullptr, *dy = nullptr, *dh = nullptr,
        *dz = nullptr, *loss_part = nullptr;
};

namespace nys {
namespace {

constexpr int MT = 16;  // 16 x 16 output tile per block

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// Z (B x O) = X (B x I) W^T + b with W (O x I) BF16; H = act(Z) (act = GELU if gelu, else identity)
__global__ void mlp_linear_fwd_kernel(const float* __restrict__ X, const __nv_bfloat16* __restrict__ W,
                                      const __nv_bfloat16* __restrict__ bias, int B, int I, int O,
                                      float* __restrict__ Z, float* __restrict__ H, int gelu) {
  __shared__ float xs[MT][MT + 1];
  __shared__ float ws[MT][MT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * MT + ty;   // batch index
  const int col = blockIdx.x * MT + tx;   // output unit
  float acc = 0.f;
  for (int k0 = 0; k0 < I; k0 += MT) {
    const int kx = k0 + tx;
    xs[ty][tx] = (row < B && kx < I) ? X[(int64_t)row * I + kx] : 0.f;
    const int wr = blockIdx.x * MT + ty, kw = k0 + tx;
    ws[ty][tx] = (wr < O && kw < I) ? __bfloat162float(W[(int64_t)wr * I + kw]) : 0.f;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < MT; ++kk) acc = fmaf(xs[ty][kk], ws[tx][kk], acc);
    __syncthreads();
  }
  if (row < B && col < O) {
    const float z = acc + __bfloat162float(bias[col]);
    if (Z) Z[(int64_t)row * O + col] = z;
    H[(int64_t)row * O + col] = gelu ? gelu_f(z) : z;
  }
}

// dX (B x I) = dZ (B x O) W (O x I)
__global__ void mlp_linear_bwd_data_kernel(const float* __restrict__ dZ, const __nv_bfloat16* __restrict__ W, int B,
                                           int I, int O, float* __restrict__ dX) {
  __shared__ float ds[MT][MT + 1];
  __shared__ float ws[MT][MT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * MT + ty;   // batch
  const int col = blockIdx.x * MT + tx;   // input unit
  float acc = 0.f;
  for (int k0 = 0; k0 < O; k0 += MT) {
    const int kd = k0 + tx;
    ds[ty][tx] = (row < B && kd < O) ? dZ[(int64_t)row * O + kd] : 0.f;
    const int kw = k0 + ty;
    ws[ty][tx] = (kw < O && col < I) ? __bfloat162float(W[(int64_t)kw * I + col]) : 0.f;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < MT; ++kk) acc = fmaf(ds[ty][kk], ws[kk][tx], acc);
    __syncthreads();
  }
  if (row < B && col < I) dX[(int64_t)row * I + col] = acc;
}

// dW (O x I) = dZ^T X, db = sum_b dZ  (thread per weight; fixed order over the batch)
__global__ void mlp_linear_bwd_weight_kernel(const float* __restrict__ dZ, const float* __restrict__ X, int B, int I,
                                             int O, float* __restrict__ dW, float* __restrict__ db) {
  __shared__ float ds[MT][MT + 1];
  __shared__ float xs[MT][MT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int o = blockIdx.y * MT + ty;
  const int i = blockIdx.x * MT + tx;
  float acc = 0.f, accb = 0.f;
  for (int b0 = 0; b0 < B; b0 += MT) {
    const int bb = b0 + tx;
    ds[ty][tx] = (o < O && bb < B) ? dZ[(int64_t)bb * O + o] : 0.f;       // ds[o][b]
    const int bx = b0 + ty;
    xs[ty][tx] = (bx < B && i < I) ? X[(int64_t)bx * I + i] : 0.f;        // xs[b][i]
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < MT; ++kk) {
      acc = fmaf(ds[ty][kk], xs[kk][tx], acc);
      accb += ds[ty][kk];
    }
    __syncthreads();
  }
  if (o < O && i < I) dW[(int64_t)o * I + i] = acc;
  if (o < O && blockIdx.x == 0 && tx == 0) db[o] = accb;
}

__global__ void mlp_gelu_bwd_kernel(int64_t n, const float* __restrict__ dH, const float* __restrict__ Z,
                                    float* __restrict__ dZ) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dZ[i] = dH[i] * gelu_grad_f(Z[i]);
}

// dY = 2 (Y - T) / (B O); per-block partials of the squared error
__global__ void mlp_mse_kernel(int64_t n, const float* __restrict__ Y, const float* __restrict__ T, float scale,
                               float* __restrict__ dY, float* __restrict__ part) {
  __shared__ double sh[kVecThreads / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float r = Y[i] - T[i];
    dY[i] = 2.f * r * scale;
    acc += (double)r * r;
  }
  acc = block_sum<kVecThreads>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = (float)acc;
}

__global__ void mlp_adam_kernel(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, __nv_bfloat16* __restrict__ w16, float lr, float b1, float b2,
                                float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    w16[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void mlp_to_bf16_kernel(int64_t n, const float* __restrict__ w, __nv_bfloat16* __restrict__ w16) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w16[i] = __float2bfloat16_rn(w[i]);
}

unsigned grid1(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(4096, (n + 255) / 256)); }

struct Layout {
  int64_t W1, b1, W2, b2, W3, b3, total;
};
Layout layout(int ni, int nh, int no) {
  Layout L;
  L.W1 = 0;
  L.b1 = L.W1 + (int64_t)nh * ni;
  L.W2 = L.b1 + nh;
  L.b2 = L.W2 + (int64_t)nh * nh;
  L.W3 = L.b2 + nh;
  L.b3 = L.W3 + (int64_t)no * nh;
  L.total = L.b3 + no;
  return L;
}

cudaError_t ensure_batch(nys_mlp_s* M, int B) {
  if (B <= M->cap) return cudaSuccess;
  float** bufs[] = {&M->z1, &M->h1, &M->z2, &M->h2, &M->y, &M->dy, &M->dh, &M->dz};
  for (float** p : bufs)
    if (*p) {
      cudaFree(*p);
      *p = nullptr;
    }
  if (M->loss_part) cudaFree(M->loss_part);
  const int64_t nh = M->n_hid, no = M->n_out, ni = M->n_in;
  const int64_t wide = std::max(nh, std::max(no, ni));
  NYS_CUDA_TRY(cudaMalloc(&M->z1, B * nh * 4));
  NYS_CUDA_TRY(cudaMalloc(&M->h1, B * nh * 4));
  NYS_CUDA_TRY(cudaMalloc(&M->z2, B * nh * 4));
  NYS_CUDA_TRY(cudaMalloc(&M->h2, B * nh * 4));
  NYS_CUDA_TRY(cudaMalloc(&M->y, B * no * 4));
  NYS_CUDA_TRY(cudaMalloc(&M->dy, B * no * 4));
  NYS_CUDA_TRY(cudaMalloc(&M->dh, B * wide * 4));
  NYS_CUDA_TRY(cudaMalloc(&M->dz, B * wide * 4));
  NYS_CUDA_TRY(cudaMalloc(&M->loss_part, 4096 * 4));
  M->cap = B;
  return cudaSuccess;
}

}  // namespace

// Forward on device buffers (usable inside a graph capture: no allocation, no sync).
// Hidden activations go to h1, h2 (B x n_hid); output to Y (B x n_out).
cudaError_t mlp_forward_dev(const nys_mlp_s* M, const float* X, int B, float* z1, float* h1, float* z2, float* h2,
                            float* Y, cudaStream_t st) {
  const Layout L = layout(M->n_in, M->n_hid, M->n_out);
  const dim3 blk(MT, MT);
  const int ni = M->n_in, nh = M->n_hid, no = M->n_out;
  count_launch();
  mlp_linear_fwd_kernel<<<dim3((nh + MT - 1) / MT, (B + MT - 1) / MT), blk, 0, st>>>(X, M->w16 + L.W1, M->w16 + L.b1,
                                                                                     B, ni, nh, z1, h1, 1);
  count_launch();
  mlp_linear_fwd_kernel<<<dim3((nh + MT - 1) / MT, (B + MT - 1) / MT), blk, 0, st>>>(h1, M->w16 + L.W2, M->w16 + L.b2,
                                                                                     B, nh, nh, z2, h2, 1);
  count_launch();
  mlp_linear_fwd_kernel<<<dim3((no + MT - 1) / MT, (B + MT - 1) / MT), blk, 0, st>>>(h2, M->w16 + L.W3, M->w16 + L.b3,
                                                                                     B, nh, no, nullptr, Y, 0);
  return cudaGetLastError();
}

int mlp_dims(const nys_mlp_s* M, int* ni, int* nh, int* no) {
  *ni = M->n_in;
  *nh = M->n_hid;
  *no = M->n_out;
  return 0;
}

// loss and gradient (into M->grad) for a batch
static cudaError_t mlp_loss_grad(nys_mlp_s* M, const float* X, const float* T, int B, float* loss_h, cudaStream_t st) {
  NYS_CUDA_TRY(ensure_batch(M, B));
  const Layout L = layout(M->n_in, M->n_hid, M->n_out);
  const int ni = M->n_in, nh = M->n_hid, no = M->n_out;
  const dim3 blk(MT, MT);
  NYS_CUDA_TRY(mlp_forward_dev(M, X, B, M->z1, M->h1, M->z2, M->h2, M->y, st));
  const int64_t ny = (int64_t)B * no;
  const unsigned gm = std::min<unsigned>(grid1(ny), 4096);
  count_launch();
  mlp_mse_kernel<<<gm, kVecThreads, 0, st>>>(ny, M->y, T, 1.f / (float)ny, M->dy, M->loss_part);
  // layer 3
  count_launch();
  mlp_linear_bwd_weight_kernel<<<dim3((nh + MT - 1) / MT, (no + MT - 1) / MT), blk, 0, st>>>(
      M->dy, M->h2, B, nh, no, M->grad + L.W3, M->grad + L.b3);
  count_launch();
  mlp_linear_bwd_data_kernel<<<dim3((nh + MT - 1) / MT, (B + MT - 1) / MT), blk, 0, st>>>(M->dy, M->w16 + L.W3, B, nh,
                                                                                          no, M->dh);
  count_launch();
  mlp_gelu_bwd_kernel<<<grid1((int64_t)B * nh), 256, 0, st>>>((int64_t)B * nh, M->dh, M->z2, M->dz);
  // layer 2
  count_launch();
  mlp_linear_bwd_weight_kernel<<<dim3((nh + MT - 1) / MT, (nh + MT - 1) / MT), blk, 0, st>>>(
      M->dz, M->h1, B, nh, nh, M->grad + L.W2, M->grad + L.b2);
  count_launch();
  mlp_linear_bwd_data_kernel<<<dim3((nh + MT - 1) / MT, (B + MT - 1) / MT), blk, 0, st>>>(M->dz, M->w16 + L.W2, B, nh,
                                                                                          nh, M->dh);
  count_launch();
  mlp_gelu_bwd_kernel<<<grid1((int64_t)B * nh), 256, 0, st>>>((int64_t)B * nh, M->dh, M->z1, M->dz);
  // layer 1
  count_launch();
  mlp_linear_bwd_weight_kernel<<<dim3((ni + MT - 1) / MT, (nh + MT - 1) / MT), blk, 0, st>>>(
      M->dz, X, B, ni, nh, M->grad + L.W1, M->grad + L.b1);
  NYS_CUDA_TRY(cudaGetLastError());
  if (loss_h) {
    std::vector<float> part(gm);
    NYS_CUDA_TRY(cudaMemcpyAsync(part.data(), M->loss_part, gm * 4, cudaMemcpyDeviceToHost, st));
    NYS_CUDA_TRY(cudaStreamSynchronize(st));
    double s = 0.0;
    for (float p : part) s += p;
    *loss_h = (float)(s / (double)ny);
  }
  return cudaSuccess;
}

}  // namespace nys

namespace {
nys_status st_of(cudaError_t e) {
  return e == cudaSuccess ? NYS_OK : (e == cudaErrorMemoryAllocation ? NYS_ENOMEM : NYS_ECUDA);
}
}  // namespace

extern "C" {

nys_status nys_mlp_create(int32_t n_in, int32_t n_hid, int32_t n_out, const float* init_params, nys_mlp* out) {
  if (!out || n_in < 1 || n_hid < 1 || n_out < 1 || n_in > 4096 || n_hid > 4096 || n_out > 4096 || !init_params)
    return NYS_EINVAL;
  *out = nullptr;
  nys_mlp_s* M = new (std::nothrow) nys_mlp_s();
  if (!M) return NYS_ENOMEM;
  M->n_in = n_in;
  M->n_hid = n_hid;
  M->n_out = n_out;
  M->n_params = layout(n_in, n_hid, n_out).total;
  const size_t n = (size_t)M->n_params;
  cudaError_t e = cudaMalloc(&M->w32, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&M->w16, n * 2);
  if (e == cudaSuccess) e = cudaMalloc(&M->grad, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&M->m, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&M->v, n * 4);
  if (e == cudaSuccess) e = cudaMemcpy(M->w32, init_params, n * 4, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemset(M->m, 0, n * 4);
  if (e == cudaSuccess) e = cudaMemset(M->v, 0, n * 4);
  if (e == cudaSuccess) {
    count_launch();
    mlp_to_bf16_kernel<<<grid1((int64_t)n), 256>>>((int64_t)n, M->w32, M->w16);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    nys_mlp_destroy(M);
    return st_of(e);
  }
  *out = M;
  return NYS_OK;
}

nys_status nys_mlp_forward(nys_mlp M, const float* X, int32_t B, float* Y, void* stream) {
  if (!M || !X || !Y || B < 1) return NYS_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = ensure_batch(M, B);
  if (e == cudaSuccess) e = mlp_forward_dev(M, X, B, M->z1, M->h1, M->z2, M->h2, Y, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return st_of(e);
}

nys_status nys_mlp_grad(nys_mlp M, const float* X, const float* T, int32_t B, float* grad_out, float* loss,
                        void* stream) {
  if (!M || !X || !T || B < 1) return NYS_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = mlp_loss_grad(M, X, T, B, loss, st);
  if (e == cudaSuccess && grad_out)
    e = cudaMemcpyAsync(grad_out, M->grad, (size_t)M->n_params * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return st_of(e);
}

nys_status nys_mlp_train_step(nys_mlp M, const float* X, const float* T, int32_t B, float lr, float* loss,
                              void* stream) {
  if (!M || !X || !T || B < 1 || !(lr > 0.f)) return NYS_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = mlp_loss_grad(M, X, T, B, loss, st);
  if (e == cudaSuccess) {
    M->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)M->step), c2 = 1.f - std::pow(b2, (float)M->step);
    count_launch();
    mlp_adam_kernel<<<grid1(M->n_params), 256, 0, st>>>(M->n_params, M->w32, M->grad, M->m, M->v, M->w16, lr, b1, b2,
                                                         1e-8f, c1, c2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return st_of(e);
}

nys_status nys_mlp_get_params(nys_mlp M, float* out, int64_t* n_params, void* stream) {
  if (!M) return NYS_EINVAL;
  if (n_params) *n_params = M->n_params;
  if (!out) return NYS_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(out, M->w32, (size_t)M->n_params * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return st_of(e);
}

void nys_mlp_destroy(nys_mlp M) {
  if (!M) return;
  float* bufs[] = {M->w32, M->grad, M->m, M->v, M->z1, M->h1, M->z2, M->h2, M->y, M->dy, M->dh, M->dz, M->loss_part};
  for (float* p : bufs)
    if (p) cudaFree(p);
  if (M->w16) cudaFree(M->w16);
  delete M;
}

}  // extern "C"
