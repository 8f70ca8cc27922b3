// The learned warm start for the occupation optimisation: a 3-layer MLP
// (features -> H tanh -> H tanh -> outputs) with BF16 weights and FP32
// arithmetic, trained and evaluated by these kernels.  The paper has no
// learned part; the network predicts the converged angles of one pairing
// subspace from its features (see onopt.cu for the features).
//
// Parameters (FP32 master copy, one array): W1 [H][F], b1 [H], W2 [H][H], b2 [H],
// W3 [O][H], b3 [O].  The matrices are also kept as BF16 (the values every
// product uses); biases, activations, gradients and the Adam moments are FP32.
// Loss: mean squared error over the batch and outputs.  Adam (beta1 0.9,
// beta2 0.999, eps 1e-8) with decoupled weight decay on the matrices.
// Every reduction over the batch is a fixed-order loop, so a step is bitwise
// reproducible.
#include "common.cuh"

#include <cuda_bf16.h>
#include <stdlib.h>

struct donof_mlp {
  int F, H, O, max_batch;
  cudaStream_t stream;
  long long nparam;
  float* P;        // master parameters
  float* G;        // gradients
  float* M;        // Adam first moments
  float* V;        // Adam second moments
  __nv_bfloat16* Wb;  // BF16 copies of W1, W2, W3 (same offsets as in P, biases unused)
  float *mean, *inv_std;
  float *X, *T, *Z0, *A1, *A2, *Y, *dY, *dZ2, *dZ1, *partial, *loss;
  long long step;
};

namespace donof {

static long long mlp_off(const donof_mlp* n, int which) {
  const long long F = n->F, H = n->H, O = n->O;
  const long long o[7] = {0, H * F, H * F + H, H * F + H + H * H, H * F + 2 * H + H * H, H * F + 2 * H + H * H + O * H,
                          H * F + 2 * H + H * H + O * H + O};
  return o[which];
}

__global__ void mlp_normalize_kernel(const float* X, int B, int F, const float* mean, const float* inv_std,
                                     float* Z) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)B * F) return;
  const int f = (int)(i % F);
  Z[i] = (X[i] - mean[f]) * inv_std[f];
}

// out[b][o] = act(bias[o] + sum_i W[o][i] in[b][i]); thread per (b, o).
__global__ void mlp_dense_kernel(const float* in, int B, int nin, const __nv_bfloat16* W, const float* bias,
                                 int nout, float* out, int act) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)B * nout) return;
  const int b = (int)(t / nout), o = (int)(t % nout);
  const float* x = in + (size_t)b * nin;
  const __nv_bfloat16* w = W + (size_t)o * nin;
  float z = bias[o];
  for (int i = 0; i < nin; ++i) z = fmaf(__bfloat162float(w[i]), x[i], z);
  out[t] = act ? tanhf(z) : z;
}

// dY = 2 (Y - T) / (B O); per-block partial sums of (Y - T)^2.
__global__ void mlp_loss_kernel(const float* Y, const float* T, long long n, float* dY, float* partial) {
  __shared__ float red[256];
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float d = 0.f;
  if (i < n) {
    d = Y[i] - T[i];
    dY[i] = 2.f * d / (float)n;
  }
  red[threadIdx.x] = d * d;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void mlp_sum_kernel(const float* partial, int n, float scale, float* out) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += 256) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] * scale;
}

// dZprev[b][i] = (sum_o dZ[b][o] W[o][i]) (1 - A[b][i]^2): back through a tanh layer.
__global__ void mlp_backprop_kernel(const float* dZ, int B, int nout, const __nv_bfloat16* W, int nin, const float* A,
                                    float* dZprev) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)B * nin) return;
  const int b = (int)(t / nin), i = (int)(t % nin);
  const float* d = dZ + (size_t)b * nout;
  float s = 0.f;
  for (int o = 0; o < nout; ++o) s = fmaf(d[o], __bfloat162float(W[(size_t)o * nin + i]), s);
  const float a = A[t];
  dZprev[t] = s * (1.f - a * a);
}

// gW[o][i] = sum_b dZ[b][o] Ain[b][i] (i < nin); gb[o] = sum_b dZ[b][o] (i == nin).
__global__ void mlp_wgrad_kernel(const float* dZ, int B, int nout, const float* Ain, int nin, float* gW, float* gb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nout * (nin + 1)) return;
  const int o = t / (nin + 1), i = t % (nin + 1);
  float s = 0.f;
  if (i < nin) {
    for (int b = 0; b < B; ++b) s = fmaf(dZ[(size_t)b * nout + o], Ain[(size_t)b * nin + i], s);
    gW[(size_t)o * nin + i] = s;
  } else {
    for (int b = 0; b < B; ++b) s += dZ[(size_t)b * nout + o];
    gb[o] = s;
  }
}

// Adam on every parameter; weight decay on [0, n_mat) ranges flagged by is_mat; BF16 refresh.
__global__ void mlp_adam_kernel(float* P, const float* G, float* M, float* V, __nv_bfloat16* Wb, long long n,
                                long long o1, long long o2, long long o3, long long o4, long long o5, float lr,
                                float c1, float c2, float wd) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool mat = (i < o1) || (i >= o2 && i < o3) || (i >= o4 && i < o5);
  const float g = G[i];
  const float m = 0.9f * M[i] + 0.1f * g;
  const float v = 0.999f * V[i] + 0.001f * g * g;
  M[i] = m;
  V[i] = v;
  float upd = lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
  if (mat) upd += lr * wd * P[i];
  const float p = P[i] - upd;
  P[i] = p;
  if (mat) Wb[i] = __float2bfloat16_rn(p);
}

__global__ void mlp_to_bf16_kernel(const float* P, __nv_bfloat16* Wb, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) Wb[i] = __float2bfloat16_rn(P[i]);
}

static unsigned int blocks(long long n, int t = 256) { return (unsigned int)((n + t - 1) / t); }

static int mlp_forward_dev(donof_mlp* n, const float* X, int B) {
  cudaStream_t s = n->stream;
  mlp_normalize_kernel<<<blocks((long long)B * n->F), 256, 0, s>>>(X, B, n->F, n->mean, n->inv_std, n->Z0);
  mlp_dense_kernel<<<blocks((long long)B * n->H), 256, 0, s>>>(n->Z0, B, n->F, n->Wb + mlp_off(n, 0),
                                                              n->P + mlp_off(n, 1), n->H, n->A1, 1);
  mlp_dense_kernel<<<blocks((long long)B * n->H), 256, 0, s>>>(n->A1, B, n->H, n->Wb + mlp_off(n, 2),
                                                              n->P + mlp_off(n, 3), n->H, n->A2, 1);
  mlp_dense_kernel<<<blocks((long long)B * n->O), 256, 0, s>>>(n->A2, B, n->H, n->Wb + mlp_off(n, 4),
                                                              n->P + mlp_off(n, 5), n->O, n->Y, 0);
  return cudaGetLastError() == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}

static int mlp_backward_dev(donof_mlp* n, const float* T, int B) {
  cudaStream_t s = n->stream;
  const long long ny = (long long)B * n->O;
  const unsigned int nb = blocks(ny);
  mlp_loss_kernel<<<nb, 256, 0, s>>>(n->Y, T, ny, n->dY, n->partial);
  mlp_sum_kernel<<<1, 256, 0, s>>>(n->partial, (int)nb, 1.f / (float)ny, n->loss);
  mlp_wgrad_kernel<<<blocks((long long)n->O * (n->H + 1)), 256, 0, s>>>(n->dY, B, n->O, n->A2, n->H,
                                                                         n->G + mlp_off(n, 4), n->G + mlp_off(n, 5));
  mlp_backprop_kernel<<<blocks((long long)B * n->H), 256, 0, s>>>(n->dY, B, n->O, n->Wb + mlp_off(n, 4), n->H, n->A2,
                                                                  n->dZ2);
  mlp_wgrad_kernel<<<blocks((long long)n->H * (n->H + 1)), 256, 0, s>>>(n->dZ2, B, n->H, n->A1, n->H,
                                                                         n->G + mlp_off(n, 2), n->G + mlp_off(n, 3));
  mlp_backprop_kernel<<<blocks((long long)B * n->H), 256, 0, s>>>(n->dZ2, B, n->H, n->Wb + mlp_off(n, 2), n->H, n->A1,
                                                                  n->dZ1);
  mlp_wgrad_kernel<<<blocks((long long)n->H * (n->F + 1)), 256, 0, s>>>(n->dZ1, B, n->H, n->Z0, n->F,
                                                                         n->G + mlp_off(n, 0), n->G + mlp_off(n, 1));
  return cudaGetLastError() == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}

static bool is_dev(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int stage_in(donof_mlp* n, float* dst, const float* src, long long count) {
  if (cudaMemcpyAsync(dst, src, count * sizeof(float), is_dev(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      n->stream) != cudaSuccess)
    return DONOF_RI_E_CUDA;
  return DONOF_RI_OK;
}

static int stage_out(donof_mlp* n, float* dst, const float* src, long long count) {
  const bool dev = is_dev(dst);
  if (cudaMemcpyAsync(dst, src, count * sizeof(float), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      n->stream) != cudaSuccess)
    return DONOF_RI_E_CUDA;
  if (!dev && cudaStreamSynchronize(n->stream) != cudaSuccess) return DONOF_RI_E_CUDA;
  return DONOF_RI_OK;
}

int mlp_forward_device(donof_mlp* n, const float* dX, int B, float** dY) {
  if (!n || B < 1 || B > n->max_batch) return DONOF_RI_E_ARG;
  int rc = mlp_forward_dev(n, dX, B);
  *dY = n->Y;
  return rc;
}

int mlp_shape(const donof_mlp* n, int* F, int* O) {
  *F = n->F;
  *O = n->O;
  return DONOF_RI_OK;
}

}  // namespace donof

using namespace donof;

extern "C" int donof_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, void* stream, donof_mlp** out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 4096 || n_hidden > 4096 || n_out > 4096 ||
      max_batch < 1 || max_batch > (1 << 24))
    return DONOF_RI_E_ARG;
  donof_mlp* n = (donof_mlp*)calloc(1, sizeof(donof_mlp));
  if (!n) return DONOF_RI_E_OOM;
  n->F = n_in;
  n->H = n_hidden;
  n->O = n_out;
  n->max_batch = max_batch;
  n->stream = (cudaStream_t)stream;
  n->nparam = mlp_off(n, 6);
  const long long B = max_batch;
  float** fl[] = {&n->P, &n->G, &n->M, &n->V};
  bool ok = true;
  for (float** f : fl) ok = ok && cudaMalloc((void**)f, n->nparam * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&n->Wb, n->nparam * sizeof(__nv_bfloat16)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&n->mean, n_in * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&n->inv_std, n_in * sizeof(float)) == cudaSuccess;
  const long long sizes[] = {B * n_in, B * n_out, B * n_in, B * n_hidden, B * n_hidden, B * n_out,
                             B * n_out, B * n_hidden, B * n_hidden, (B * n_out + 255) / 256 + 1, 1};
  float** bufs[] = {&n->X, &n->T, &n->Z0, &n->A1, &n->A2, &n->Y, &n->dY, &n->dZ2, &n->dZ1, &n->partial, &n->loss};
  for (int i = 0; i < 11; ++i) ok = ok && cudaMalloc((void**)bufs[i], sizes[i] * sizeof(float)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    donof_mlp_destroy(n);
    return DONOF_RI_E_OOM;
  }
  cudaMemsetAsync(n->P, 0, n->nparam * sizeof(float), n->stream);
  cudaMemsetAsync(n->M, 0, n->nparam * sizeof(float), n->stream);
  cudaMemsetAsync(n->V, 0, n->nparam * sizeof(float), n->stream);
  cudaMemsetAsync(n->Wb, 0, n->nparam * sizeof(__nv_bfloat16), n->stream);
  cudaMemsetAsync(n->mean, 0, n_in * sizeof(float), n->stream);
  // inv_std = 1
  {
    float* ones = (float*)malloc(n_in * sizeof(float));
    for (int i = 0; i < n_in; ++i) ones[i] = 1.f;
    cudaMemcpy(n->inv_std, ones, n_in * sizeof(float), cudaMemcpyHostToDevice);
    free(ones);
  }
  if (cudaStreamSynchronize(n->stream) != cudaSuccess) {
    donof_mlp_destroy(n);
    return DONOF_RI_E_CUDA;
  }
  *out = n;
  return DONOF_RI_OK;
}

extern "C" long long donof_mlp_param_count(const donof_mlp* n) { return n ? n->nparam : -1; }

extern "C" int donof_mlp_set_params(donof_mlp* n, const float* params) {
  if (!n || !params) return DONOF_RI_E_ARG;
  int rc = stage_in(n, n->P, params, n->nparam);
  if (rc) return rc;
  cudaMemsetAsync(n->M, 0, n->nparam * sizeof(float), n->stream);
  cudaMemsetAsync(n->V, 0, n->nparam * sizeof(float), n->stream);
  mlp_to_bf16_kernel<<<blocks(n->nparam), 256, 0, n->stream>>>(n->P, n->Wb, n->nparam);
  n->step = 0;
  return cudaStreamSynchronize(n->stream) == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}

extern "C" int donof_mlp_get_params(donof_mlp* n, float* params) {
  if (!n || !params) return DONOF_RI_E_ARG;
  return stage_out(n, params, n->P, n->nparam);
}

extern "C" int donof_mlp_set_normalization(donof_mlp* n, const float* mean, const float* inv_std) {
  if (!n || !mean || !inv_std) return DONOF_RI_E_ARG;
  int rc = stage_in(n, n->mean, mean, n->F);
  if (rc) return rc;
  rc = stage_in(n, n->inv_std, inv_std, n->F);
  if (rc) return rc;
  return cudaStreamSynchronize(n->stream) == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}

extern "C" int donof_mlp_forward(donof_mlp* n, const float* X, int batch, float* Y) {
  if (!n || !X || !Y || batch < 1 || batch > n->max_batch) return DONOF_RI_E_ARG;
  int rc = stage_in(n, n->X, X, (long long)batch * n->F);
  if (rc) return rc;
  if ((rc = mlp_forward_dev(n, n->X, batch))) return rc;
  return stage_out(n, Y, n->Y, (long long)batch * n->O);
}

extern "C" int donof_mlp_loss_grad(donof_mlp* n, const float* X, const float* T, int batch, float* loss, float* grads) {
  if (!n || !X || !T || batch < 1 || batch > n->max_batch) return DONOF_RI_E_ARG;
  int rc = stage_in(n, n->X, X, (long long)batch * n->F);
  if (rc) return rc;
  if ((rc = stage_in(n, n->T, T, (long long)batch * n->O))) return rc;
  if ((rc = mlp_forward_dev(n, n->X, batch))) return rc;
  if ((rc = mlp_backward_dev(n, n->T, batch))) return rc;
  if (loss && (rc = stage_out(n, loss, n->loss, 1))) return rc;
  if (grads && (rc = stage_out(n, grads, n->G, n->nparam))) return rc;
  return cudaStreamSynchronize(n->stream) == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}

extern "C" int donof_mlp_train_step(donof_mlp* n, const float* X, const float* T, int batch, float lr,
                                    float weight_decay, float* loss) {
  if (!n || !X || !T || batch < 1 || batch > n->max_batch || !(lr >= 0.f) || !(weight_decay >= 0.f))
    return DONOF_RI_E_ARG;
  int rc = stage_in(n, n->X, X, (long long)batch * n->F);
  if (rc) return rc;
  if ((rc = stage_in(n, n->T, T, (long long)batch * n->O))) return rc;
  if ((rc = mlp_forward_dev(n, n->X, batch))) return rc;
  if ((rc = mlp_backward_dev(n, n->T, batch))) return rc;
  n->step += 1;
  const double c1 = 1.0 / (1.0 - pow(0.9, (double)n->step)), c2 = 1.0 / (1.0 - pow(0.999, (double)n->step));
  mlp_adam_kernel<<<blocks(n->nparam), 256, 0, n->stream>>>(n->P, n->G, n->M, n->V, n->Wb, n->nparam, mlp_off(n, 1),
                                                            mlp_off(n, 2), mlp_off(n, 3), mlp_off(n, 4), mlp_off(n, 5),
                                                            lr, (float)c1, (float)c2, weight_decay);
  if (cudaGetLastError() != cudaSuccess) return DONOF_RI_E_CUDA;
  if (loss) return stage_out(n, loss, n->loss, 1);
  return DONOF_RI_OK;
}

extern "C" int donof_mlp_destroy(donof_mlp* n) {
  if (!n) return DONOF_RI_E_ARG;
  void* bufs[] = {n->P, n->G, n->M, n->V, n->Wb, n->mean, n->inv_std, n->X, n->T, n->Z0, n->A1, n->A2,
                  n->Y, n->dY, n->dZ2, n->dZ1, n->partial, n->loss};
  for (void* b : bufs)
    if (b) cudaFree(b);
  free(n);
  return DONOF_RI_OK;
}
