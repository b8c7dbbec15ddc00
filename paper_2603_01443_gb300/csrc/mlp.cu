// A small fully connected FP32 network for the learned stage-time planner:
// forward pass, mean-squared-error gradient, backward pass and Adam updates
// as hand-written kernels.  Layers l = 0..L-1 map dims[l] -> dims[l+1];
// hidden layers use ReLU, the last layer is linear.  Parameters are packed
// per layer as W_l (dims[l+1] x dims[l], row-major) followed by b_l.
//
// Sizes are tiny (inputs of a few features, widths of 64, a few thousand
// samples), so each kernel maps one thread to one output element and the
// whole training run is a sequence of launches on one stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace cc {
namespace {

constexpr int kMaxLayers = 8;
constexpr int kMaxWidth = 1024;

// y[n, o] = act(b[o] + sum_i x[n, i] W[o, i])
__global__ void dense_forward(const float* __restrict__ x, const float* __restrict__ W,
                              const float* __restrict__ b, float* __restrict__ y, int64_t n,
                              int din, int dout, int relu) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * dout) return;
  const int64_t s = e / dout;
  const int o = (int)(e - s * dout);
  const float* xr = x + s * din;
  const float* wr = W + (int64_t)o * din;
  float acc = b[o];
  for (int i = 0; i < din; ++i) acc = fmaf(xr[i], wr[i], acc);
  y[e] = relu ? fmaxf(acc, 0.f) : acc;
}

// g = 2 (y - t) / (n * dout) (gradient of the mean squared error), and the
// per-sample squared errors for the loss.
__global__ void mse_grad(const float* __restrict__ y, const float* __restrict__ t,
                         float* __restrict__ g, float* __restrict__ sq, int64_t count) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float d = y[e] - t[e];
  g[e] = 2.f * d / (float)count;
  sq[e] = d * d;
}

// dx[n, i] = sum_o dy[n, o] W[o, i], then masked by the ReLU of x's layer
// (x > 0) when mask is set.
__global__ void dense_backward_input(const float* __restrict__ dy, const float* __restrict__ W,
                                     const float* __restrict__ x, float* __restrict__ dx,
                                     int64_t n, int din, int dout, int mask) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * din) return;
  const int64_t s = e / din;
  const int i = (int)(e - s * din);
  const float* dyr = dy + s * dout;
  float acc = 0.f;
  for (int o = 0; o < dout; ++o) acc = fmaf(dyr[o], W[(int64_t)o * din + i], acc);
  dx[e] = (mask && x[e] <= 0.f) ? 0.f : acc;
}

// dW[o, i] = sum_n dy[n, o] x[n, i];  db[o] = sum_n dy[n, o].  One block per
// (o, i) pair (i = din stands for the bias), threads stride over samples.
__global__ void dense_backward_weights(const float* __restrict__ dy, const float* __restrict__ x,
                                       float* __restrict__ dW, float* __restrict__ db, int64_t n,
                                       int din, int dout) {
  const int o = blockIdx.x / (din + 1), i = blockIdx.x % (din + 1);
  float acc = 0.f;
  for (int64_t s = threadIdx.x; s < n; s += blockDim.x)
    acc += dy[s * dout + o] * (i < din ? x[s * din + i] : 1.f);
  __shared__ float red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (i < din) dW[(int64_t)o * din + i] = red[0];
    else db[o] = red[0];
  }
}

// Adam (Kingma and Ba, 2015) with bias correction.
__global__ void adam_update(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int64_t count, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.f - b1) * gi;
  const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void sum_kernel(const float* __restrict__ a, int64_t count, float* __restrict__ out) {
  __shared__ float red[256];
  float acc = 0.f;
  for (int64_t e = threadIdx.x; e < count; e += blockDim.x) acc += a[e];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] / (float)count;
}

unsigned blocks(int64_t count) { return (unsigned)((count + 255) / 256); }

struct Layout {
  std::vector<int64_t> w_off, b_off;  // parameter offsets (floats)
  int64_t n_params = 0;
  std::vector<int64_t> act_off;  // activations a_0 = x (not stored), a_1..a_L
  int64_t act_floats = 0;
  int max_width = 0;
};

cc_status layout(const int32_t* dims, int n_layers, int64_t n, Layout& L) {
  if (!dims) return fail(CC_EINVAL, "dims is NULL");
  if (n_layers < 1 || n_layers > kMaxLayers) return fail(CC_ERANGE, "n_layers must be in 1..8");
  if (n < 0) return fail(CC_EINVAL, "n < 0");
  for (int l = 0; l <= n_layers; ++l)
    if (dims[l] < 1 || dims[l] > kMaxWidth) return fail(CC_ERANGE, "layer width must be in 1..1024");
  L = Layout();
  for (int l = 0; l < n_layers; ++l) {
    L.w_off.push_back(L.n_params);
    L.n_params += (int64_t)dims[l + 1] * dims[l];
    L.b_off.push_back(L.n_params);
    L.n_params += dims[l + 1];
  }
  L.act_off.push_back(0);
  for (int l = 1; l <= n_layers; ++l) {
    L.act_off.push_back(L.act_floats);
    L.act_floats += n * dims[l];
  }
  for (int l = 0; l <= n_layers; ++l) L.max_width = std::max(L.max_width, (int)dims[l]);
  return CC_OK;
}

// Workspace (floats): activations a_1..a_L, two gradient buffers of
// n * max_width, squared errors n * dims[L], parameter gradients, 1 loss slot.
int64_t work_floats(const Layout& L, int64_t n, int out_dim) {
  return L.act_floats + 2 * n * L.max_width + n * out_dim + L.n_params + 1;
}

cc_status check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return CC_OK;
}

void forward(const int32_t* dims, int n_layers, const float* params, const float* x, int64_t n,
             float* acts, const Layout& L, cudaStream_t s) {
  const float* in = x;
  for (int l = 0; l < n_layers; ++l) {
    float* out = acts + L.act_off[l + 1];
    dense_forward<<<blocks(n * dims[l + 1]), 256, 0, s>>>(
        in, params + L.w_off[l], params + L.b_off[l], out, n, dims[l], dims[l + 1],
        l + 1 < n_layers ? 1 : 0);
    in = out;
  }
}

}  // namespace
}  // namespace cc

using namespace cc;

extern "C" uint64_t cc_mlp_work_bytes(const int32_t* dims, int32_t n_layers, int64_t n) {
  Layout L;
  if (layout(dims, n_layers, n, L) != CC_OK) return 0;
  return (uint64_t)work_floats(L, n, dims[n_layers]) * sizeof(float);
}

extern "C" int64_t cc_mlp_param_count(const int32_t* dims, int32_t n_layers) {
  Layout L;
  if (layout(dims, n_layers, 0, L) != CC_OK) return -1;
  return L.n_params;
}

extern "C" cc_status cc_mlp_forward(const int32_t* dims, int32_t n_layers, const float* params,
                                    const float* x, int64_t n, float* y, float* work,
                                    uint64_t work_bytes, void* stream) {
  Layout L;
  cc_status st = layout(dims, n_layers, n, L);
  if (st != CC_OK) return st;
  if (!params || !x || !y || !work) return fail(CC_EINVAL, "NULL buffer");
  if (work_bytes < (uint64_t)work_floats(L, n, dims[n_layers]) * sizeof(float))
    return fail(CC_EBUFSIZE, "MLP workspace too small");
  if (n == 0) return CC_OK;
  st = check_device();
  if (st != CC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  forward(dims, n_layers, params, x, n, work, L, s);
  const cudaError_t e = cudaMemcpyAsync(y, work + L.act_off[n_layers],
                                        sizeof(float) * n * dims[n_layers],
                                        cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
  return check_launch("MLP forward");
}

extern "C" cc_status cc_mlp_train(const int32_t* dims, int32_t n_layers, float* params,
                                  float* adam_m, float* adam_v, const float* x, const float* t,
                                  int64_t n, int32_t epochs, float lr, float* loss, float* work,
                                  uint64_t work_bytes, void* stream) {
  Layout L;
  cc_status st = layout(dims, n_layers, n, L);
  if (st != CC_OK) return st;
  if (!params || !adam_m || !adam_v || !x || !t || !work) return fail(CC_EINVAL, "NULL buffer");
  if (n < 1) return fail(CC_EINVAL, "no training samples");
  if (epochs < 0) return fail(CC_EINVAL, "epochs < 0");
  if (!(lr > 0.f) || !std::isfinite(lr)) return fail(CC_EINVAL, "lr must be positive");
  const int out_dim = dims[n_layers];
  if (work_bytes < (uint64_t)work_floats(L, n, out_dim) * sizeof(float))
    return fail(CC_EBUFSIZE, "MLP workspace too small");
  st = check_device();
  if (st != CC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  float* acts = work;
  float* g0 = acts + L.act_floats;
  float* g1 = g0 + n * L.max_width;
  float* sq = g1 + n * L.max_width;
  float* grads = sq + n * out_dim;
  float* loss_tmp = grads + L.n_params;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < epochs; ++ep) {
    forward(dims, n_layers, params, x, n, acts, L, s);
    const float* y = acts + L.act_off[n_layers];
    mse_grad<<<blocks(n * out_dim), 256, 0, s>>>(y, t, g0, sq, n * out_dim);
    sum_kernel<<<1, 256, 0, s>>>(sq, n * out_dim, loss ? loss + ep : loss_tmp);
    float* dy = g0;
    float* dx = g1;
    for (int l = n_layers - 1; l >= 0; --l) {
      const float* xin = l == 0 ? x : acts + L.act_off[l];
      dense_backward_weights<<<(unsigned)(dims[l + 1] * (dims[l] + 1)), 256, 0, s>>>(
          dy, xin, grads + L.w_off[l], grads + L.b_off[l], n, dims[l], dims[l + 1]);
      if (l > 0) {
        dense_backward_input<<<blocks(n * dims[l]), 256, 0, s>>>(
            dy, params + L.w_off[l], xin, dx, n, dims[l], dims[l + 1], 1);
        std::swap(dy, dx);
      }
    }
    const float c1 = 1.f - std::pow(b1, (float)(ep + 1)), c2 = 1.f - std::pow(b2, (float)(ep + 1));
    adam_update<<<blocks(L.n_params), 256, 0, s>>>(params, grads, adam_m, adam_v, L.n_params, lr,
                                                   b1, b2, eps, c1, c2);
  }
  return check_launch("MLP training");
}
