// Fourier-neural-operator surrogate of the split-step solver: forward,
// backward, loss and Adam.  Every contraction runs on BF16 tensor cores with
// FP32 accumulation: the truncated DFTs in streaming passes of their own
// (dft_x_kernel, dft_y_kernel, idft_y_kernel), the spectral layers' inverse
// DFT along x with the 1x1 convolution in the tcgen05 layer kernel, the rest
// on the batched GEMM; pointwise work is fused into those kernels or runs in
// small kernels of its own.
//
// Network (channels C, grid s x s, kept modes ky in {0..m-1} u {s-m..s-1},
// kx in {0..m-1}, Nm = 2m * m modes):
//   v0 = P a + pb
//   z_l = Spec_l(v_l) + W_l v_l + b_l,  v_{l+1} = gelu(z_l) (identity after the last layer)
//   Spec(v) = (1/s^2) sum w_kx Re(U e^{+i th}), U = R V (per mode), V = sum v e^{-i th}
//   h = gelu(Q1 v_L + q1b),  (phi, dr, di) = Q2 h + q2b,
//   out = psi e^{-i phi} + (dr + i di)  with psi = a[0] + i a[1]
// The truncated DFTs are separable real GEMMs: along x with an s x 2m
// cos/sin matrix, along y per plane with a 4m x s block matrix.  Mode mixing
// is a batch of Nm complex C x C GEMMs written as four real ones.
// Activations are planar [B][C][s][s] FP32; modes are [B][C][re|im][Nm].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sn.h"
#include "sn_internal.h"

using namespace sn;

namespace {
constexpr double kPi = 3.14159265358979323846;
typedef long long ll;
}  // namespace

struct sn_fno_s {
  int s = 0, ci = 0, C = 0, m = 0, L = 0, J = 0, Bmax = 0;
  ll P = 0, Nm = 0, nparams = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
  ll off_P = 0, off_pb = 0, off_Q1 = 0, off_q1b = 0, off_Q2 = 0, off_q2b = 0;
  std::vector<ll> off_R, off_W, off_b;
  float *ExF = nullptr, *ExFw = nullptr, *EyA = nullptr, *EyB = nullptr;
  float *EyIre = nullptr, *EyIim = nullptr, *WxI = nullptr, *WxI1 = nullptr;
  __nv_bfloat16* EyAB = nullptr;  // [EyA | EyB] rounded to BF16, 4m x 2s (dft_y_kernel)
  __nv_bfloat16* EyI = nullptr;   // [EyIre ; EyIim] rounded to BF16, 2s x 4m (idft_y_kernel)
  float *a = nullptr, *A1 = nullptr, *Uh = nullptr, *B1 = nullptr, *g1 = nullptr, *h = nullptr;
  float *out = nullptr, *dout = nullptr, *dv = nullptr, *dv2 = nullptr, *dz = nullptr, *dh = nullptr;
  float *yh = nullptr, *dy = nullptr;  // head channels (phi, dr, di) and their gradient
  // how a spectral layer's inverse DFT along x, 1x1 convolution, bias and
  // activation run (sn_fno_set_layer_form), and the fused form's status word
  int layer_form = SN_FNO_LAYER_GEMMS;  // sn_fno_create takes the fused form where it applies
  int* status = nullptr;
  float *GU = nullptr, *GV = nullptr, *work = nullptr;
  std::vector<float*> v, z, Vh;
  double* norms = nullptr;  // per sample (||out - t||^2, ||t||^2), then the B gradient scales
  double* loss_part = nullptr;  // per sample and chunk, the two partial sums
  double* chan_part = nullptr;  // channel-sum partials [max channels][kChanParts]
  int lastB = 0;
  int sms = 1;  // the device's SM count (grids of the persistent kernels)
  ll work_floats = 0;
  std::vector<void*> allocs;
};

namespace {

sn_status ffail(sn_status st, const std::string& m) {
  set_thread_error(m.c_str());
  return st;
}
sn_status fcuda(cudaError_t e, const char* what) {
  return ffail(e == cudaErrorMemoryAllocation ? SN_ENOMEM : SN_ECUDA,
               std::string("fno: ") + what + ": " + cudaGetErrorString(e));
}
#define FCHK(call)                                  \
  do {                                              \
    cudaError_t _e = (call);                        \
    if (_e != cudaSuccess) return fcuda(_e, #call); \
  } while (0)

template <typename T>
cudaError_t falloc(sn_fno f, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) return e;
  f->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return cudaSuccess;
}

// ---- pointwise kernels --------------------------------------------------------

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) +
         x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

// bias_act over rows of P values: about 8 blocks per row, at least one
inline dim3 rows_grid(ll rows, ll P) {
  const ll per = std::max<ll>(1, std::min<ll>(8, (P + 1023) / 1024));
  return dim3((unsigned)per, (unsigned)rows);
}

inline unsigned blocks_for(ll n) {
  const ll b = (n + 255) / 256;
  return (unsigned)(b < 8192 ? b : 8192);
}

// z[b][c][p] += bias[c]; v = gelu(z) (act) or z.  Block (x, r) covers a span of
// row r = b C + c (P contiguous values), four values per thread step.
__global__ void bias_act_kernel(float* z, const float* bias, float* v, ll C, ll P, int act) {
  const ll r = blockIdx.y;
  const float bc = bias[r % C];
  float* zr = z + r * P;
  float* vr = v != nullptr ? v + r * P : nullptr;
  const ll span = (P + gridDim.x - 1) / gridDim.x;
  const ll p0 = blockIdx.x * span, p1 = min(P, p0 + span);
  if ((P & 3) == 0 && (span & 3) == 0) {
    for (ll p = p0 + 4 * threadIdx.x; p < p1; p += 4 * blockDim.x) {
      float4 x = *reinterpret_cast<float4*>(zr + p);
      x.x += bc; x.y += bc; x.z += bc; x.w += bc;
      *reinterpret_cast<float4*>(zr + p) = x;
      if (vr != nullptr) {
        if (act) x = make_float4(gelu(x.x), gelu(x.y), gelu(x.z), gelu(x.w));
        *reinterpret_cast<float4*>(vr + p) = x;
      }
    }
  } else {
    for (ll p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
      const float x = zr[p] + bc;
      zr[p] = x;
      if (vr != nullptr) vr[p] = act ? gelu(x) : x;
    }
  }
}

__global__ void gelu_bwd_kernel(const float* dv, const float* z, float* dz, ll n) {
  const ll n4 = n / 4;
  for (ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x; i < n4; i += (ll)gridDim.x * blockDim.x) {
    const float4 d = reinterpret_cast<const float4*>(dv)[i], x = reinterpret_cast<const float4*>(z)[i];
    reinterpret_cast<float4*>(dz)[i] =
        make_float4(d.x * gelu_grad(x.x), d.y * gelu_grad(x.y), d.z * gelu_grad(x.z), d.w * gelu_grad(x.w));
  }
  for (ll i = 4 * n4 + blockIdx.x * (ll)blockDim.x + threadIdx.x; i < n; i += (ll)gridDim.x * blockDim.x)
    dz[i] = dv[i] * gelu_grad(z[i]);
}

// out = psi e^{-i phi} + (dr + i di): psi = (a[b][0], a[b][1]), (phi, dr, di) = y[b][0..2]
__global__ void head_kernel(const float* a, const float* y, float* out, ll ci, ll P, ll n) {
  for (ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x; i < n; i += (ll)gridDim.x * blockDim.x) {
    const ll b = i / P, p = i - b * P;
    const float pr = a[b * ci * P + p], pi = a[b * ci * P + P + p];
    const float* yy = y + b * 3 * P + p;
    float s, c;
    sincosf(yy[0], &s, &c);
    out[b * 2 * P + p] = pr * c + pi * s + yy[P];
    out[b * 2 * P + P + p] = pi * c - pr * s + yy[2 * P];
  }
}

// dy = (dout_r rot_i - dout_i rot_r, dout_r, dout_i) with rot = psi e^{-i phi}
__global__ void head_bwd_kernel(const float* a, const float* y, const float* dout, float* dy, ll ci,
                                ll P, ll n) {
  for (ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x; i < n; i += (ll)gridDim.x * blockDim.x) {
    const ll b = i / P, p = i - b * P;
    const float pr = a[b * ci * P + p], pi = a[b * ci * P + P + p];
    float s, c;
    sincosf(y[b * 3 * P + p], &s, &c);
    const float rr = pr * c + pi * s, ri = pi * c - pr * s;
    const float gr = dout[b * 2 * P + p], gi = dout[b * 2 * P + P + p];
    dy[b * 3 * P + p] = gr * ri - gi * rr;
    dy[b * 3 * P + P + p] = gr;
    dy[b * 3 * P + 2 * P + p] = gi;
  }
}

// The lift, 1x1 from the input channels: v[b][c][p] = bias[c] + sum_i
// W[c][i] a[b][i][p] (i in order), FP32.  Each thread takes four neighbouring
// pixels of one sample (P is a multiple of 4) and writes every channel; W and
// the bias sit in shared memory.
constexpr int kLiftMaxIn = 16;
__global__ void lift_kernel(const float* a, const float* W, const float* bias, float* v, int ci,
                            int C, ll P, ll B) {
  extern __shared__ float lift_sm[];
  float* Ws = lift_sm;       // [C][ci]
  float* bs = lift_sm + C * ci;
  for (int k = threadIdx.x; k < C * ci; k += blockDim.x) Ws[k] = W[k];
  for (int k = threadIdx.x; k < C; k += blockDim.x) bs[k] = bias[k];
  __syncthreads();
  const ll P4 = P / 4, n4 = B * P4;
  for (ll q = blockIdx.x * (ll)blockDim.x + threadIdx.x; q < n4; q += (ll)gridDim.x * blockDim.x) {
    const ll b = q / P4, p = 4 * (q - b * P4);
    float4 x[kLiftMaxIn];
#pragma unroll
    for (int i = 0; i < kLiftMaxIn; ++i)
      if (i < ci) x[i] = *reinterpret_cast<const float4*>(a + (b * ci + i) * P + p);
    for (int c = 0; c < C; ++c) {
      float4 acc = make_float4(bs[c], bs[c], bs[c], bs[c]);
#pragma unroll
      for (int i = 0; i < kLiftMaxIn; ++i) {
        if (i < ci) {
          const float w = Ws[c * ci + i];
          acc.x = fmaf(w, x[i].x, acc.x);
          acc.y = fmaf(w, x[i].y, acc.y);
          acc.z = fmaf(w, x[i].z, acc.z);
          acc.w = fmaf(w, x[i].w, acc.w);
        }
      }
      *reinterpret_cast<float4*>(v + (b * C + c) * P + p) = acc;
    }
  }
}

// The projection's last 1x1 and the head, per pixel: y[k] = b2[k] + sum_j
// Q2[k][j] h[b][j][p] (j in order, k = phi, dr, di), kept in yh for the
// backward, then out = psi e^{-i phi} + (dr + i di) as head_kernel, FP32.
__global__ void proj_head_kernel(const float* h, const float* Q2, const float* b2, const float* a,
                                 float* yh, float* out, int J, int ci, ll P, ll B) {
  extern __shared__ float head_sm[];
  for (int k = threadIdx.x; k < 3 * J; k += blockDim.x) head_sm[k] = Q2[k];
  __syncthreads();
  const ll P4 = P / 4, n4 = B * P4;
  for (ll q = blockIdx.x * (ll)blockDim.x + threadIdx.x; q < n4; q += (ll)gridDim.x * blockDim.x) {
    const ll b = q / P4, p = 4 * (q - b * P4);
    float4 y[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) y[k] = make_float4(b2[k], b2[k], b2[k], b2[k]);
    const float* hb = h + b * J * P + p;
    for (int j = 0; j < J; ++j) {
      const float4 x = *reinterpret_cast<const float4*>(hb + (ll)j * P);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float w = head_sm[k * J + j];
        y[k].x = fmaf(w, x.x, y[k].x);
        y[k].y = fmaf(w, x.y, y[k].y);
        y[k].z = fmaf(w, x.z, y[k].z);
        y[k].w = fmaf(w, x.w, y[k].w);
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) *reinterpret_cast<float4*>(yh + (b * 3 + k) * P + p) = y[k];
    const float4 pr = *reinterpret_cast<const float4*>(a + b * ci * P + p);
    const float4 pi = *reinterpret_cast<const float4*>(a + b * ci * P + P + p);
    float4 o_r, o_i;
    float s, c;
    sincosf(y[0].x, &s, &c); o_r.x = pr.x * c + pi.x * s + y[1].x; o_i.x = pi.x * c - pr.x * s + y[2].x;
    sincosf(y[0].y, &s, &c); o_r.y = pr.y * c + pi.y * s + y[1].y; o_i.y = pi.y * c - pr.y * s + y[2].y;
    sincosf(y[0].z, &s, &c); o_r.z = pr.z * c + pi.z * s + y[1].z; o_i.z = pi.z * c - pr.z * s + y[2].z;
    sincosf(y[0].w, &s, &c); o_r.w = pr.w * c + pi.w * s + y[1].w; o_i.w = pi.w * c - pr.w * s + y[2].w;
    *reinterpret_cast<float4*>(out + b * 2 * P + p) = o_r;
    *reinterpret_cast<float4*>(out + b * 2 * P + P + p) = o_i;
  }
}

// The backward of the projection's last 1x1 through the GELU before it:
// dh[b][j][p] = GELU'(g1[b][j][p]) sum_k Q2[k][j] dy[b][k][p], FP32.
__global__ void proj_dh_kernel(const float* dy, const float* Q2, const float* g1, float* dh, int J,
                               ll P, ll B) {
  const ll P4 = P / 4, n4 = B * (ll)J * P4;
  for (ll q = blockIdx.x * (ll)blockDim.x + threadIdx.x; q < n4; q += (ll)gridDim.x * blockDim.x) {
    const ll row = q / P4, p = 4 * (q - row * P4);  // row = b J + j
    const ll b = row / J;
    const int j = (int)(row - b * J);
    const float w0 = Q2[j], w1 = Q2[J + j], w2 = Q2[2 * J + j];
    const float4 d0 = *reinterpret_cast<const float4*>(dy + (b * 3) * P + p);
    const float4 d1 = *reinterpret_cast<const float4*>(dy + (b * 3 + 1) * P + p);
    const float4 d2 = *reinterpret_cast<const float4*>(dy + (b * 3 + 2) * P + p);
    const float4 z = *reinterpret_cast<const float4*>(g1 + row * P + p);
    float4 r;
    r.x = fmaf(w2, d2.x, fmaf(w1, d1.x, w0 * d0.x)) * gelu_grad(z.x);
    r.y = fmaf(w2, d2.y, fmaf(w1, d1.y, w0 * d0.y)) * gelu_grad(z.y);
    r.z = fmaf(w2, d2.z, fmaf(w1, d1.z, w0 * d0.z)) * gelu_grad(z.z);
    r.w = fmaf(w2, d2.w, fmaf(w1, d1.w, w0 * d0.w)) * gelu_grad(z.w);
    *reinterpret_cast<float4*>(dh + row * P + p) = r;
  }
}

// out[c] = sum_b sum_p X[b][c][p] in a fixed order: block (c, j) sums span j of
// every row of channel c into part[c][j] (FP64), then one thread per channel
// adds its parts.
constexpr int kChanParts = 64;
__global__ void channel_part_kernel(const float* X, ll B, ll C, ll P, double* part) {
  const ll c = blockIdx.x;
  const int j = blockIdx.y;
  const ll span = (P + kChanParts - 1) / kChanParts;
  const ll p0 = j * span, p1 = min(P, p0 + span);
  // per-thread sums in FP32 (at most a few hundred terms; FP64 adds are slow
  // on this GPU), combined across the block in FP64
  float sf = 0.f;
  for (ll b = 0; b < B; ++b) {
    const float* row = X + (b * C + c) * P;
    for (ll p = p0 + threadIdx.x; p < p1; p += blockDim.x) sf += row[p];
  }
  const double s = sf;
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[c * kChanParts + j] = red[0];
}
__global__ void channel_final_kernel(const double* part, ll C, float* out) {
  const ll c = blockIdx.x * (ll)blockDim.x + threadIdx.x;
  if (c >= C) return;
  double s = 0.0;
  for (int j = 0; j < kChanParts; ++j) s += part[c * kChanParts + j];
  out[c] = (float)s;
}

// per sample b: norms[2b] = ||out_b - t_b||^2, norms[2b+1] = ||t_b||^2, in
// FP64.  kLossParts blocks per sample each sum one contiguous chunk (per
// thread, then a tree over the block) into part[b][j]; loss_final_kernel adds
// the parts in order and stores the gradient's scale 1 / (B ||out_b - t_b||
// ||t_b||) (0 where a norm is 0) after the 2B norms.
constexpr int kLossParts = 64;

__global__ void loss_parts_kernel(const float* out, const float* t, ll n_per, double* part) {
  const ll b = blockIdx.x;
  const int j = blockIdx.y;
  const ll span = (n_per + kLossParts - 1) / kLossParts;
  const ll i0 = j * span, i1 = min(n_per, i0 + span);
  double d2 = 0.0, t2 = 0.0;
  for (ll i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double o = out[b * n_per + i], tt = t[b * n_per + i];
    d2 += (o - tt) * (o - tt);
    t2 += tt * tt;
  }
  __shared__ double r1[256], r2[256];
  r1[threadIdx.x] = d2;
  r2[threadIdx.x] = t2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      r1[threadIdx.x] += r1[threadIdx.x + w];
      r2[threadIdx.x] += r2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * (b * kLossParts + j)] = r1[0];
    part[2 * (b * kLossParts + j) + 1] = r2[0];
  }
}

__global__ void loss_final_kernel(const double* part, ll B, double* norms) {
  const ll b = blockIdx.x * (ll)blockDim.x + threadIdx.x;
  if (b >= B) return;
  double d2 = 0.0, t2 = 0.0;
  for (int j = 0; j < kLossParts; ++j) {
    d2 += part[2 * (b * kLossParts + j)];
    t2 += part[2 * (b * kLossParts + j) + 1];
  }
  norms[2 * b] = d2;
  norms[2 * b + 1] = t2;
  const double den = (double)B * sqrt(d2) * sqrt(t2);
  norms[2 * B + b] = den > 0.0 ? 1.0 / den : 0.0;
}

// dout = (out - t) / (B ||out_b - t_b|| ||t_b||), the scale taken per sample
__global__ void loss_grad_kernel(const float* out, const float* t, const double* norms, ll n_per,
                                 ll B, float* dout) {
  for (ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x; i < B * n_per;
       i += (ll)gridDim.x * blockDim.x) {
    const ll b = i / n_per;
    dout[i] = (float)(((double)out[i] - (double)t[i]) * norms[2 * B + b]);
  }
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, ll n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x; i < n; i += (ll)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// X[b] = (re, im, f0, f1, f2) planes from interleaved psi[b] and feats[b][3]
__global__ void pack_kernel(const float2* psi, const float* feats, int nf, float* X, ll P, ll n) {
  for (ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x; i < n; i += (ll)gridDim.x * blockDim.x) {
    const ll b = i / P, p = i - b * P;
    const float2 z = psi[i];
    float* x = X + b * (2 + nf) * P + p;
    x[0] = z.x;
    x[P] = z.y;
    for (int k = 0; k < nf; ++k) x[(2 + k) * P] = feats[b * nf + k];
  }
}

// X[b] = (re a, im a, re c, im c, f0, f1, ...) planes from interleaved a[b], c[b]
// and feats[b][nf]
__global__ void pack2_kernel(const float2* a, const float2* c, const float* feats, int nf, float* X,
                             ll P, ll n) {
  for (ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x; i < n; i += (ll)gridDim.x * blockDim.x) {
    const ll b = i / P, p = i - b * P;
    const float2 za = a[i], zc = c[i];
    float* x = X + b * (4 + nf) * P + p;
    x[0] = za.x;
    x[P] = za.y;
    x[2 * P] = zc.x;
    x[3 * P] = zc.y;
    for (int k = 0; k < nf; ++k) x[(4 + k) * P] = feats[b * nf + k];
  }
}

__global__ void unpack_kernel(const float* Y, float2* psi, ll P, ll n) {
  for (ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x; i < n; i += (ll)gridDim.x * blockDim.x) {
    const ll b = i / P, p = i - b * P;
    psi[i] = make_float2(Y[b * 2 * P + p], Y[b * 2 * P + P + p]);
  }
}

// out[b] = sum_p |psi[b][p]|^2 (FP64, one block per state, fixed order)
__global__ void mass_kernel(const float2* psi, ll P, double* out) {
  const ll b = blockIdx.x;
  double s = 0.0;
  for (ll p = threadIdx.x; p < P; p += blockDim.x) {
    const float2 z = psi[b * P + p];
    s += (double)z.x * z.x + (double)z.y * z.y;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] = red[0];
}

// ---- truncated DFT along y of whole planes --------------------------------------
// V (4m x m) = [EyA | EyB] (4m x 2s) [A1re ; A1im] (2s x m) for every plane: the
// two per-plane GEMMs of the y transform as one product with K = 2s.  The
// 4m x 2s table, rounded to BF16 once (dfty_table_kernel), is copied into
// shared memory once per CTA with 16-byte loads; each plane's A1 (s x 2m
// FP32) is read once, rounded to BF16 like the GEMM's operands and stored
// [k][n]; the next plane's A1 is loaded into registers while the current one
// is multiplied.  Two groups of m / 4 warps, one warp per 16 rows of V in each,
// take the two halves of K (the EyA and the EyB products); the second group's
// sums go through shared memory to the first, which adds them and stores V.
// NT n-tiles of 8 modes each (mma.sync m16n8k16, FP32 accumulation).  Row
// strides: the table's 2s + 8 and the plane operand's dfty_ns(m) BF16 values,
// both an odd multiple of 4 words modulo 8, which keeps the fragment loads on
// 32 banks.
constexpr int kDftyMaxLoads = 8;  // float4 of a plane per thread: s / 32 <= 8

__host__ __device__ constexpr int dfty_ns(int m) {
  return ((((m + 7) / 8) * 4) % 8 == 4 ? ((m + 7) / 8) * 8 : ((m + 7) / 8) * 8 + 8);
}
inline size_t dfty_smem(int s, int m) {
  return sizeof(__nv_bfloat16) * ((size_t)4 * m * (2 * s + 8) + (size_t)2 * s * dfty_ns(m)) +
         sizeof(float) * (size_t)(m / 4) * 32 * 4 * ((m + 7) / 8);  // the second group's sums
}

__device__ __forceinline__ void mma_16x8x16_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                                 unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned bf16_pair(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// [EyA | EyB] (4m rows of s + s) rounded to BF16 into one 4m x 2s table
__global__ void dfty_table_kernel(const float* EyA, const float* EyB, __nv_bfloat16* T, int s,
                                  int m) {
  const ll n = (ll)4 * m * 2 * s;
  for (ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x; i < n; i += (ll)gridDim.x * blockDim.x) {
    const ll r = i / (2 * s), k = i - r * (2 * s);
    T[i] = __float2bfloat16_rn(k < s ? EyA[r * s + k] : EyB[r * s + (k - s)]);
  }
}

template <int NT>
__global__ void __launch_bounds__(512) dft_y_kernel(const __nv_bfloat16* __restrict__ EyAB,
                                                    const float* __restrict__ A1,
                                                    float* __restrict__ V, int s, int m, ll planes,
                                                    ll vstride) {
  extern __shared__ __align__(16) unsigned char dfty_sm[];
  const int KS = 2 * s + 8, NS = dfty_ns(m);
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(dfty_sm);  // [4m][KS]
  __nv_bfloat16* Bs = As + (size_t)4 * m * KS;                      // [2s][NS]
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, gid = lane >> 2, tig = lane & 3;
  {
    // the table in 16-byte chunks of 8 values (s / 4 per row; rows of KS
    // values keep them 16-byte aligned), eight loads in flight a thread
    const int cpr = s / 4, nch = 4 * m * cpr;
    const uint4* src = reinterpret_cast<const uint4*>(EyAB);
    for (int i0 = tid; i0 < nch; i0 += 8 * nth) {
      uint4 w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (i0 + u * nth < nch) w[u] = src[i0 + u * nth];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * nth;
        if (i < nch) {
          const int r = i / cpr, c = i - r * cpr;
          *reinterpret_cast<uint4*>(As + r * KS + 8 * c) = w[u];
        }
      }
    }
  }
  const int nq = s * m / 2;  // float4 of one plane's A1
  float4 pre[kDftyMaxLoads];
  auto load = [&](ll pl) {
    const float4* src = reinterpret_cast<const float4*>(A1 + pl * (ll)s * 2 * m);
#pragma unroll
    for (int i = 0; i < kDftyMaxLoads; ++i) {
      const int q = tid + nth * i;
      if (q < nq) pre[i] = src[q];
    }
  };
  ll p = blockIdx.x;
  if (p < planes) load(p);
  for (; p < planes; p += gridDim.x) {
    __syncthreads();  // the previous plane's fragment reads (and the table's writes) are done
#pragma unroll
    for (int i = 0; i < kDftyMaxLoads; ++i) {
      const int q = tid + nth * i;
      if (q < nq) {
        const int e = 4 * q, y = e / (2 * m), c = e - y * (2 * m);
        const int row = c < m ? y : s + y, col = c < m ? c : c - m;
        uint2 w;
        w.x = bf16_pair(__float2bfloat16_rn(pre[i].x), __float2bfloat16_rn(pre[i].y));
        w.y = bf16_pair(__float2bfloat16_rn(pre[i].z), __float2bfloat16_rn(pre[i].w));
        *reinterpret_cast<uint2*>(Bs + row * NS + col) = w;
      }
    }
    __syncthreads();
    if (p + gridDim.x < planes) load(p + gridDim.x);
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[j][r] = 0.f;
    const int nwm = m / 4;                            // warps per half of K
    const int kh = warp / nwm, mt = warp - kh * nwm;  // half of K, row tile
    const int r0 = mt * 16 + gid;
    for (int kk = kh * s; kk < kh * s + s; kk += 16) {
      unsigned af[4];
      af[0] = *reinterpret_cast<const unsigned*>(As + r0 * KS + kk + 2 * tig);
      af[1] = *reinterpret_cast<const unsigned*>(As + (r0 + 8) * KS + kk + 2 * tig);
      af[2] = *reinterpret_cast<const unsigned*>(As + r0 * KS + kk + 2 * tig + 8);
      af[3] = *reinterpret_cast<const unsigned*>(As + (r0 + 8) * KS + kk + 2 * tig + 8);
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const __nv_bfloat16* b = Bs + (kk + 2 * tig) * NS + 8 * j + gid;
        mma_16x8x16_bf16(acc[j], af, bf16_pair(b[0], b[NS]), bf16_pair(b[8 * NS], b[9 * NS]));
      }
    }
    // the EyB half's sums to the EyA half (the next plane's writes of Bs come
    // after the barrier at the top of the loop, so red is free again by then)
    float* red = reinterpret_cast<float*>(Bs + (size_t)2 * s * NS) + (size_t)(mt * 32 + lane) * 4 * NT;
    if (kh == 1) {
#pragma unroll
      for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int r = 0; r < 4; ++r) red[4 * j + r] = acc[j][r];
    }
    __syncthreads();
    if (kh == 1) continue;
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[j][r] += red[4 * j + r];
    float* out = V + p * vstride;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int col = 8 * j + 2 * tig;
      if (col < m) {
        out[(ll)r0 * m + col] = acc[j][0];
        out[(ll)(r0 + 8) * m + col] = acc[j][2];
      }
      if (col + 1 < m) {
        out[(ll)r0 * m + col + 1] = acc[j][1];
        out[(ll)(r0 + 8) * m + col + 1] = acc[j][3];
      }
    }
  }
}

// The truncated DFT along x of every row: A1 (rows x 2m) = X (rows x s) Ex
// (s x 2m).  X is read once, straight into the A fragments (FP32 pairs
// rounded to BF16 in registers, as the GEMM rounds its operands); Ex is
// rounded to BF16 into shared memory once per CTA ([n][k], stride s + 8, an
// odd multiple of 4 words modulo 8 for the fragment loads).  Each warp takes
// 16 rows at a time with NT2 = 2m / 8 n-tiles (mma.sync m16n8k16, FP32
// accumulation in the GEMM's k order).
constexpr int kDftxThreads = 256;

inline size_t dftx_smem(int s, int m) { return sizeof(__nv_bfloat16) * (size_t)2 * m * (s + 8); }

template <int NT2>
__global__ void __launch_bounds__(kDftxThreads) dft_x_kernel(const float* __restrict__ X,
                                                             const float* __restrict__ Ex,
                                                             float* __restrict__ A1, int s, int m,
                                                             ll rows) {
  extern __shared__ __align__(16) unsigned char dftx_sm[];
  const int KS = s + 8, N2 = 2 * m;
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(dftx_sm);  // [2m][KS]
  const int tid = threadIdx.x, nth = kDftxThreads;
  const int lane = tid & 31, warp = tid >> 5, gid = lane >> 2, tig = lane & 3;
  for (int i = tid; i < s * N2; i += nth) {
    const int k = i / N2, n = i - k * N2;
    Bs[n * KS + k] = __float2bfloat16_rn(Ex[i]);
  }
  __syncthreads();
  const ll tiles = rows / 16;
  const int wpb = nth / 32;
  for (ll t = (ll)blockIdx.x * wpb + warp; t < tiles; t += (ll)gridDim.x * wpb) {
    const float* x0 = X + (t * 16 + gid) * (ll)s + 2 * tig;  // row gid of the tile
    const float* x1 = x0 + 8 * (ll)s;                         // row gid + 8
    float acc[NT2][4];
#pragma unroll
    for (int j = 0; j < NT2; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[j][r] = 0.f;
#pragma unroll 4
    for (int kk = 0; kk < s; kk += 16) {
      const float2 a00 = __ldcs(reinterpret_cast<const float2*>(x0 + kk));
      const float2 a10 = __ldcs(reinterpret_cast<const float2*>(x1 + kk));
      const float2 a01 = __ldcs(reinterpret_cast<const float2*>(x0 + kk + 8));
      const float2 a11 = __ldcs(reinterpret_cast<const float2*>(x1 + kk + 8));
      const unsigned af[4] = {bf16_pair(__float2bfloat16_rn(a00.x), __float2bfloat16_rn(a00.y)),
                              bf16_pair(__float2bfloat16_rn(a10.x), __float2bfloat16_rn(a10.y)),
                              bf16_pair(__float2bfloat16_rn(a01.x), __float2bfloat16_rn(a01.y)),
                              bf16_pair(__float2bfloat16_rn(a11.x), __float2bfloat16_rn(a11.y))};
#pragma unroll
      for (int j = 0; j < NT2; ++j) {
        const __nv_bfloat16* b = Bs + (8 * j + gid) * KS + kk + 2 * tig;
        mma_16x8x16_bf16(acc[j], af, *reinterpret_cast<const unsigned*>(b),
                         *reinterpret_cast<const unsigned*>(b + 8));
      }
    }
    float* o0 = A1 + (t * 16 + gid) * (ll)N2;
    float* o1 = o0 + 8 * (ll)N2;
#pragma unroll
    for (int j = 0; j < NT2; ++j) {
      const int col = 8 * j + 2 * tig;
      *reinterpret_cast<float2*>(o0 + col) = make_float2(acc[j][0], acc[j][1]);
      *reinterpret_cast<float2*>(o1 + col) = make_float2(acc[j][2], acc[j][3]);
    }
  }
}

// The inverse DFT along y of whole planes: B1 (s x 2m, [y][re q | im q]) =
// [EyIre ; EyIim] (2s x 4m) U (4m x m) per plane, rows r < s giving the real
// parts of row y = r and rows s + y the imaginary ones.  The same scheme as
// dft_y_kernel: the 2s x 4m BF16 table resident in shared memory (row stride
// 4m + 8), each plane's modes U (4m x m FP32) read once and rounded to BF16
// ([k][n], stride dfty_ns(m)), the next plane's loaded while the current one is
// multiplied; sixteen warps take the 2s / 16 row tiles in turn.
constexpr int kIdftyThreads = 512, kIdftyMaxLoads = 2;  // m^2 float4 of U <= 2 a thread

inline size_t idfty_smem(int s, int m) {
  return sizeof(__nv_bfloat16) * ((size_t)2 * s * (4 * m + 8) + (size_t)4 * m * dfty_ns(m));
}

// [top ; bottom] (two row-major blocks of n values each) rounded to BF16
__global__ void stack_bf16_kernel(const float* top, const float* bottom, __nv_bfloat16* T, ll n) {
  for (ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x; i < 2 * n; i += (ll)gridDim.x * blockDim.x)
    T[i] = __float2bfloat16_rn(i < n ? top[i] : bottom[i - n]);
}

template <int NT>
__global__ void __launch_bounds__(kIdftyThreads, 1) idft_y_kernel(const __nv_bfloat16* __restrict__ EyI,
                                                               const float* __restrict__ U,
                                                               float* __restrict__ B1, int s, int m,
                                                               ll planes, ll ustride) {
  extern __shared__ __align__(16) unsigned char idfty_sm[];
  const int KS = 4 * m + 8, NS = dfty_ns(m);
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(idfty_sm);  // [2s][KS]
  __nv_bfloat16* Bs = As + (size_t)2 * s * KS;                       // [4m][NS]
  const int tid = threadIdx.x, nth = kIdftyThreads;
  const int lane = tid & 31, warp = tid >> 5, gid = lane >> 2, tig = lane & 3;
  {
    // the table in 16-byte chunks (m / 2 per row of 4m values), eight loads
    // in flight a thread
    const int cpr = m / 2, nch = 2 * s * cpr;
    const uint4* src = reinterpret_cast<const uint4*>(EyI);
    for (int i0 = tid; i0 < nch; i0 += 8 * nth) {
      uint4 w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (i0 + u * nth < nch) w[u] = src[i0 + u * nth];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * nth;
        if (i < nch) {
          const int r = i / cpr, c = i - r * cpr;
          *reinterpret_cast<uint4*>(As + r * KS + 8 * c) = w[u];
        }
      }
    }
  }
  const int nq = m * m;  // float4 of one plane's U (4m x m)
  float4 pre[kIdftyMaxLoads];
  auto load = [&](ll pl) {
    const float4* src = reinterpret_cast<const float4*>(U + pl * ustride);
#pragma unroll
    for (int i = 0; i < kIdftyMaxLoads; ++i) {
      const int q = tid + nth * i;
      if (q < nq) pre[i] = src[q];
    }
  };
  ll p = blockIdx.x;
  if (p < planes) load(p);
  const int mtiles = 2 * s / 16;
  for (; p < planes; p += gridDim.x) {
    __syncthreads();  // the previous plane's fragment reads (and the table's writes) are done
#pragma unroll
    for (int i = 0; i < kIdftyMaxLoads; ++i) {
      const int q = tid + nth * i;
      if (q < nq) {
        const int e = 4 * q, k = e / m, c = e - k * m;
        uint2 w;
        w.x = bf16_pair(__float2bfloat16_rn(pre[i].x), __float2bfloat16_rn(pre[i].y));
        w.y = bf16_pair(__float2bfloat16_rn(pre[i].z), __float2bfloat16_rn(pre[i].w));
        *reinterpret_cast<uint2*>(Bs + k * NS + c) = w;
      }
    }
    __syncthreads();
    if (p + gridDim.x < planes) load(p + gridDim.x);
    float* out = B1 + p * (ll)s * 2 * m;
    for (int mt = warp; mt < mtiles; mt += nth / 32) {
      float acc[NT][4];
#pragma unroll
      for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[j][r] = 0.f;
      const int r0 = mt * 16 + gid;
      for (int kk = 0; kk < 4 * m; kk += 16) {
        unsigned af[4];
        af[0] = *reinterpret_cast<const unsigned*>(As + r0 * KS + kk + 2 * tig);
        af[1] = *reinterpret_cast<const unsigned*>(As + (r0 + 8) * KS + kk + 2 * tig);
        af[2] = *reinterpret_cast<const unsigned*>(As + r0 * KS + kk + 2 * tig + 8);
        af[3] = *reinterpret_cast<const unsigned*>(As + (r0 + 8) * KS + kk + 2 * tig + 8);
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          const __nv_bfloat16* b = Bs + (kk + 2 * tig) * NS + 8 * j + gid;
          mma_16x8x16_bf16(acc[j], af, bf16_pair(b[0], b[NS]), bf16_pair(b[8 * NS], b[9 * NS]));
        }
      }
      // rows r0 and r0 + 8 of the stacked product: (y, half) = (r mod s, r / s)
      float* o0 = out + (ll)(r0 % s) * 2 * m + (r0 / s) * m;
      float* o1 = out + (ll)((r0 + 8) % s) * 2 * m + ((r0 + 8) / s) * m;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int col = 8 * j + 2 * tig;
        if (col + 1 < m) {
          *reinterpret_cast<float2*>(o0 + col) = make_float2(acc[j][0], acc[j][1]);
          *reinterpret_cast<float2*>(o1 + col) = make_float2(acc[j][2], acc[j][3]);
        } else if (col < m) {
          o0[col] = acc[j][0];
          o1[col] = acc[j][2];
        }
      }
    }
  }
}

// ---- per-mode complex channel mixing ---------------------------------------
// U[b][o](mode) = sum_i V[b][i](mode) R[mode][i][o], complex, with the planar
// layout X[b][c][re/im][mode] of V and U and R[mode][i][o][re/im].  One block
// per mode; V, R and (backward) GU are rounded to BF16 on load like the GEMM
// operands, products accumulate in FP32.
__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// The forward stages the mode's R, rounded, in shared memory beside V: each R
// value serves all B samples, so it is loaded and rounded once.
__global__ void mode_mix_kernel(const float* V, const float* R, float* U, int B, int C, ll Nm) {
  extern __shared__ float mm_sm[];
  float2* Vs = reinterpret_cast<float2*>(mm_sm);  // [B][C]
  float2* Rs = Vs + B * C;                        // [C][C], rounded
  const ll mode = blockIdx.x;
  const ll is = 2 * Nm, bs = (ll)C * is;
  for (int e = threadIdx.x; e < B * C; e += blockDim.x) {
    const int b = e / C, i = e % C;
    const float* v = V + b * bs + i * is + mode;
    Vs[e] = make_float2(bf(v[0]), bf(v[Nm]));
  }
  const float2* Rm = reinterpret_cast<const float2*>(R) + mode * (ll)C * C;
  for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
    const float2 r = Rm[e];
    Rs[e] = make_float2(bf(r.x), bf(r.y));
  }
  __syncthreads();
  for (int e = threadIdx.x; e < B * C; e += blockDim.x) {
    const int b = e / C, o = e % C;
    float ar = 0.f, ai = 0.f;
    for (int i = 0; i < C; ++i) {
      const float2 x = Vs[b * C + i];
      const float2 r = Rs[i * C + o];
      const float rr = r.x, ri = r.y;
      ar = fmaf(x.x, rr, fmaf(-x.y, ri, ar));
      ai = fmaf(x.x, ri, fmaf(x.y, rr, ai));
    }
    float* u = U + b * bs + o * is + mode;
    u[0] = ar;
    u[Nm] = ai;
  }
}

// The same mixing for kMixModes consecutive modes per block: V and U of all of
// them staged in shared memory, so that the global reads and writes are runs
// of kMixModes modes (32 bytes) instead of one word per sector; R staged one
// mode at a time.  Each output is summed over i in the same order with the
// same operations as mode_mix_kernel, so the results are the same bits.
constexpr int kMixModes = 8, kMixThreads = 512;

inline size_t mode_mix8_smem(ll B, ll C) {
  return sizeof(float2) * ((size_t)2 * kMixModes * B * C + (size_t)C * C);
}

__global__ void __launch_bounds__(kMixThreads) mode_mix8_kernel(const float* V, const float* R,
                                                                float* U, int B, int C, ll Nm) {
  extern __shared__ float mm_sm[];
  const int BC = B * C;
  float2* Vs = reinterpret_cast<float2*>(mm_sm);  // [kMixModes][B][C]
  float2* Us = Vs + kMixModes * BC;               // [kMixModes][B][C]
  float2* Rs = Us + kMixModes * BC;               // [C][C], rounded
  const ll mode0 = blockIdx.x * (ll)kMixModes;
  const int nm = (int)min((ll)kMixModes, Nm - mode0);
  const ll is = 2 * Nm, bs = (ll)C * is;
  for (int e = threadIdx.x; e < BC * kMixModes; e += blockDim.x) {
    const int bi = e / kMixModes, q = e - bi * kMixModes;
    if (q < nm) {
      const int b = bi / C, i = bi - b * C;
      const float* v = V + b * bs + i * is + mode0 + q;
      Vs[q * BC + bi] = make_float2(bf(v[0]), bf(v[Nm]));
    }
  }
  for (int q = 0; q < nm; ++q) {
    __syncthreads();  // the previous mode's reads of Rs are done (and Vs is written)
    const float2* Rm = reinterpret_cast<const float2*>(R) + (mode0 + q) * (ll)C * C;
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
      const float2 r = Rm[e];
      Rs[e] = make_float2(bf(r.x), bf(r.y));
    }
    __syncthreads();
    const float2* Vq = Vs + q * BC;
    for (int e = threadIdx.x; e < BC; e += blockDim.x) {
      const int b = e / C, o = e - b * C;
      float ar = 0.f, ai = 0.f;
      for (int i = 0; i < C; ++i) {
        const float2 x = Vq[b * C + i];
        const float2 r = Rs[i * C + o];
        const float rr = r.x, ri = r.y;
        ar = fmaf(x.x, rr, fmaf(-x.y, ri, ar));
        ai = fmaf(x.x, ri, fmaf(x.y, rr, ai));
      }
      Us[q * BC + e] = make_float2(ar, ai);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < BC * kMixModes; e += blockDim.x) {
    const int bo = e / kMixModes, q = e - bo * kMixModes;
    if (q < nm) {
      const int b = bo / C, o = bo - b * C;
      float* u = U + b * bs + o * is + mode0 + q;
      const float2 w = Us[q * BC + bo];
      u[0] = w.x;
      u[Nm] = w.y;
    }
  }
}

// GR[mode][i][o] = sum_b conj(V[b][i]) GU[b][o];  GV[b][i] = sum_o conj(R[i][o]) GU[b][o]
__global__ void mode_mix_bwd_kernel(const float* V, const float* R, const float* GU, float* GR,
                                    float* GV, int B, int C, ll Nm) {
  extern __shared__ float mm_sm[];
  float2* Vs = reinterpret_cast<float2*>(mm_sm);  // [B][C]
  float2* Gs = Vs + B * C;                         // [B][C]
  float2* Rs = Gs + B * C;  // R transposed, [o][i] with row stride C + 1: the GV loop's lanes
                            // (consecutive i) then read consecutive words
  const ll mode = blockIdx.x;
  const ll is = 2 * Nm, bs = (ll)C * is;
  for (int e = threadIdx.x; e < B * C; e += blockDim.x) {
    const int b = e / C, i = e % C;
    const float* v = V + b * bs + i * is + mode;
    const float* g = GU + b * bs + i * is + mode;
    Vs[e] = make_float2(bf(v[0]), bf(v[Nm]));
    Gs[e] = make_float2(bf(g[0]), bf(g[Nm]));
  }
  const float2* Rm = reinterpret_cast<const float2*>(R) + mode * (ll)C * C;
  for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
    const float2 r = Rm[e];
    const int i = e / C, o = e % C;
    Rs[o * (C + 1) + i] = make_float2(bf(r.x), bf(r.y));
  }
  __syncthreads();
  float2* GRm = reinterpret_cast<float2*>(GR) + mode * (ll)C * C;
  for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
    const int i = e / C, o = e % C;
    float ar = 0.f, ai = 0.f;
    for (int b = 0; b < B; ++b) {
      const float2 x = Vs[b * C + i], g = Gs[b * C + o];
      ar = fmaf(x.x, g.x, fmaf(x.y, g.y, ar));   // conj(x) g
      ai = fmaf(x.x, g.y, fmaf(-x.y, g.x, ai));
    }
    GRm[e] = make_float2(ar, ai);
  }
  for (int e = threadIdx.x; e < B * C; e += blockDim.x) {
    const int b = e / C, i = e % C;
    float ar = 0.f, ai = 0.f;
    for (int o = 0; o < C; ++o) {
      const float2 r = Rs[o * (C + 1) + i], g = Gs[b * C + o];
      ar = fmaf(r.x, g.x, fmaf(r.y, g.y, ar));   // conj(r) g
      ai = fmaf(r.x, g.y, fmaf(-r.y, g.x, ai));
    }
    float* gv = GV + b * bs + i * is + mode;
    gv[0] = ar;
    gv[Nm] = ai;
  }
}

// ---- GEMM plumbing --------------------------------------------------------------

cudaError_t gemm(sn_fno f, int M, int N, int K, int Z, const float* A, ll sAz, ll sAm, ll sAk,
                 const float* B, ll sBz, ll sBk, ll sBn, float* C, ll sCz, ll sCm, ll sCn,
                 float alpha = 1.f, float beta = 0.f, const float* bias = nullptr,
                 float* C2 = nullptr, int act = 0) {
  GemmArgs g{};
  g.A = A; g.sAz = sAz; g.sAm = sAm; g.sAk = sAk;
  g.B = B; g.sBz = sBz; g.sBk = sBk; g.sBn = sBn;
  g.C = C; g.sCz = sCz; g.sCm = sCm; g.sCn = sCn; g.sCsp = 0;
  g.M = M; g.N = N; g.K = K; g.Z = Z; g.kchunk = 0;
  g.alpha = alpha; g.beta = beta;
  g.bias = bias; g.C2 = C2; g.act = act;
  return gemm_bf16(g, f->stream);
}

// dW (M x N, row-major) = sum_b dY[b] (M x P) X[b]^T (X[b] is N x P), split over K
// out[c] = sum over samples and pixels of X[b][c][p] (bias gradients)
cudaError_t channel_sum(sn_fno f, const float* X, ll B, ll C, ll P, float* out) {
  channel_part_kernel<<<dim3((unsigned)C, kChanParts), 256, 0, f->stream>>>(X, B, C, P, f->chan_part);
  channel_final_kernel<<<(unsigned)((C + 127) / 128), 128, 0, f->stream>>>(f->chan_part, C, out);
  return cudaGetLastError();
}

// Split-K width of the weight-gradient GEMMs (K = pixels): narrow enough that
// B x (P / kWgChunk) blocks fill the GPU.
constexpr int kWgChunk = 1024;

cudaError_t weight_grad(sn_fno f, const float* dY, const float* X, int B, int M, int N, float* dW) {
  const int kchunk = kWgChunk;
  const int nsplit = (int)((f->P + kchunk - 1) / kchunk);
  GemmArgs g{};
  g.A = dY; g.sAz = (ll)M * f->P; g.sAm = f->P; g.sAk = 1;
  g.B = X; g.sBz = (ll)N * f->P; g.sBk = 1; g.sBn = f->P;
  g.C = f->work; g.sCz = (ll)nsplit * M * N; g.sCm = N; g.sCn = 1; g.sCsp = (ll)M * N;
  g.M = M; g.N = N; g.K = (int)f->P; g.Z = B; g.kchunk = kchunk;
  g.alpha = 1.f; g.beta = 0.f;
  cudaError_t e = gemm_bf16(g, f->stream);
  if (e != cudaSuccess) return e;
  return reduce_sum(f->work, (ll)B * nsplit, (ll)M * N, (ll)M * N, dW, 0.f, f->stream);
}

// the whole-plane y transform (dft_y_kernel) takes m a multiple of 4 up to 32
// (one warp per 16 of the 4m rows, at most 4 n-tiles) and s a multiple of 16
// up to 256 (a plane's A1 in at most 16 float4 a thread)
bool dfty_supported(int s, int m) {
  return m % 4 == 0 && m >= 4 && m <= 32 && s % 16 == 0 && s >= 16 && s <= 256 &&
         dfty_smem(s, m) <= 200 * 1024;
}

template <int NT>
cudaError_t launch_dft_y_t(sn_fno f, ll planes, float* V) {
  const size_t smem = dfty_smem(f->s, f->m);
  const int threads = 16 * f->m;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dft_y_kernel<NT>, threads, smem);
  if (e != cudaSuccess) return e;
  const ll grid = std::min<ll>(planes, (ll)std::max(1, std::min(per_sm, 8)) * f->sms);
  dft_y_kernel<NT><<<(unsigned)grid, threads, smem, f->stream>>>(f->EyAB, f->A1, V, f->s, f->m,
                                                                 planes, 2 * f->Nm);
  return cudaGetLastError();
}

cudaError_t launch_dft_y(sn_fno f, ll planes, float* V) {
  switch ((f->m + 7) / 8) {
    case 1: return launch_dft_y_t<1>(f, planes, V);
    case 2: return launch_dft_y_t<2>(f, planes, V);
    case 3: return launch_dft_y_t<3>(f, planes, V);
    default: return launch_dft_y_t<4>(f, planes, V);
  }
}

template <int NT2>
cudaError_t launch_dft_x_t(sn_fno f, const float* X, const float* Ex, ll rows) {
  const size_t smem = dftx_smem(f->s, f->m);
  int per_sm = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dft_x_kernel<NT2>, kDftxThreads, smem);
  if (e != cudaSuccess) return e;
  const ll tiles = rows / 16, wpb = kDftxThreads / 32;
  const ll grid = std::min<ll>((tiles + wpb - 1) / wpb, (ll)std::max(1, per_sm) * f->sms);
  dft_x_kernel<NT2><<<(unsigned)grid, kDftxThreads, smem, f->stream>>>(X, Ex, f->A1, f->s, f->m, rows);
  return cudaGetLastError();
}

cudaError_t launch_dft_x(sn_fno f, const float* X, const float* Ex, ll rows) {
  switch (f->m / 4) {
    case 1: return launch_dft_x_t<1>(f, X, Ex, rows);
    case 2: return launch_dft_x_t<2>(f, X, Ex, rows);
    case 3: return launch_dft_x_t<3>(f, X, Ex, rows);
    case 4: return launch_dft_x_t<4>(f, X, Ex, rows);
    case 5: return launch_dft_x_t<5>(f, X, Ex, rows);
    case 6: return launch_dft_x_t<6>(f, X, Ex, rows);
    case 7: return launch_dft_x_t<7>(f, X, Ex, rows);
    default: return launch_dft_x_t<8>(f, X, Ex, rows);
  }
}

template <int NT>
cudaError_t launch_idft_y_t(sn_fno f, const float* U, ll planes) {
  const size_t smem = idfty_smem(f->s, f->m);
  int per_sm = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, idft_y_kernel<NT>, kIdftyThreads, smem);
  if (e != cudaSuccess) return e;
  const ll grid = std::min<ll>(planes, (ll)std::max(1, std::min(per_sm, 8)) * f->sms);
  idft_y_kernel<NT><<<(unsigned)grid, kIdftyThreads, smem, f->stream>>>(f->EyI, U, f->B1, f->s, f->m,
                                                                        planes, 2 * f->Nm);
  return cudaGetLastError();
}

cudaError_t launch_idft_y(sn_fno f, const float* U, ll planes) {
  switch ((f->m + 7) / 8) {
    case 1: return launch_idft_y_t<1>(f, U, planes);
    case 2: return launch_idft_y_t<2>(f, U, planes);
    case 3: return launch_idft_y_t<3>(f, U, planes);
    default: return launch_idft_y_t<4>(f, U, planes);
  }
}

// modes V[B][C][2][Nm] = truncated forward DFT of planes X[B][C][s][s]; Ex: s x 2m
cudaError_t dft_forward(sn_fno f, const float* X, int B, int Cn, const float* Ex, float* V) {
  const int s = f->s, m = f->m;
  const ll planes = (ll)B * Cn;
  // along x: A1 (planes*s x 2m) = X (planes*s x s) Ex (s x 2m)
  cudaError_t e = dfty_supported(s, m)
                      ? launch_dft_x(f, X, Ex, planes * s)
                      : gemm(f, (int)(planes * s), 2 * m, s, 1, X, 0, s, 1, Ex, 0, 2 * m, 1, f->A1,
                             0, 2 * m, 1);
  if (e != cudaSuccess) return e;
  // along y, per plane: V (4m x m) = EyA (4m x s) A1re (s x m) + EyB (4m x s) A1im (s x m)
  if (dfty_supported(s, m)) return launch_dft_y(f, planes, V);
  e = gemm(f, 4 * m, m, s, (int)planes, f->EyA, 0, s, 1, f->A1, (ll)s * 2 * m, 2 * m, 1, V,
           2 * f->Nm, m, 1);
  if (e != cudaSuccess) return e;
  return gemm(f, 4 * m, m, s, (int)planes, f->EyB, 0, s, 1, f->A1 + m, (ll)s * 2 * m, 2 * m, 1, V,
              2 * f->Nm, m, 1, 1.f, 1.f);
}

// the inverse DFT along y of modes U[B][C][2][Nm]: B1[B][C][s][2m], per row y
// the coefficients (re q | im q) of the inverse DFT along x
cudaError_t dft_inverse_y(sn_fno f, const float* U, int B, int Cn) {
  const int s = f->s, m = f->m;
  const ll planes = (ll)B * Cn;
  // per plane: B1re (s x m) = EyIre (s x 4m) U (4m x m); B1im likewise; B1 is [y][re|im][q]
  if (f->EyI != nullptr) return launch_idft_y(f, U, planes);
  cudaError_t e = gemm(f, s, m, 4 * m, (int)planes, f->EyIre, 0, 4 * m, 1, U, 2 * f->Nm, m, 1,
                       f->B1, (ll)s * 2 * m, 2 * m, 1);
  if (e != cudaSuccess) return e;
  return gemm(f, s, m, 4 * m, (int)planes, f->EyIim, 0, 4 * m, 1, U, 2 * f->Nm, m, 1, f->B1 + m,
              (ll)s * 2 * m, 2 * m, 1);
}

// planes Y[B][C][s][s] (=, or += with beta) from modes U[B][C][2][Nm]; Wx: 2m x s
cudaError_t dft_inverse(sn_fno f, const float* U, int B, int Cn, const float* Wx, float* Y,
                        float beta) {
  const int s = f->s, m = f->m;
  const ll planes = (ll)B * Cn;
  cudaError_t e = dft_inverse_y(f, U, B, Cn);
  if (e != cudaSuccess) return e;
  // along x: Y (planes*s x s) = B1 (planes*s x 2m) Wx (2m x s)
  return gemm(f, (int)(planes * s), s, 2 * m, 1, f->B1, 0, 2 * m, 1, Wx, 0, s, 1, Y, 0, s, 1, 1.f,
              beta);
}

// U[b][o] = sum_i R[mode][i][o] V[b][i] per mode (complex), four real GEMMs
cudaError_t mode_mix(sn_fno f, const float* V, const float* R, int B, float* U) {
  if (mode_mix8_smem(f->Bmax, f->C) <= 200 * 1024) {
    mode_mix8_kernel<<<(unsigned)((f->Nm + kMixModes - 1) / kMixModes), kMixThreads,
                       mode_mix8_smem(B, f->C), f->stream>>>(V, R, U, B, f->C, f->Nm);
    return cudaGetLastError();
  }
  const size_t sm = sizeof(float2) * ((size_t)B * f->C + (size_t)f->C * f->C);
  mode_mix_kernel<<<(unsigned)f->Nm, 256, sm, f->stream>>>(V, R, U, B, f->C, f->Nm);
  return cudaGetLastError();
}

// backward of mode_mix: GR[mode][i][o] = sum_b conj(V_i) GU_o ; GV[b][i] = sum_o conj(R_io) GU_o
cudaError_t mode_mix_bwd(sn_fno f, const float* V, const float* R, const float* GU, int B, float* GR,
                         float* GV) {
  const size_t sm = sizeof(float2) * (2 * (size_t)B * f->C + (size_t)f->C * (f->C + 1));
  mode_mix_bwd_kernel<<<(unsigned)f->Nm, 256, sm, f->stream>>>(V, R, GU, GR, GV, B, f->C, f->Nm);
  return cudaGetLastError();
}

std::vector<float> dft_matrix(int kind, int s, int m) {
  // ky list: 0..m-1, s-m..s-1 ; kx: 0..m-1
  std::vector<int> ky(2 * m);
  for (int p = 0; p < m; ++p) { ky[p] = p; ky[m + p] = s - m + p; }
  const double tw = 2.0 * kPi / s;
  const double wscale = 1.0 / ((double)s * s);
  std::vector<float> M;
  auto ang = [&](long long a, long long b) { return tw * (double)((a * b) % s); };
  if (kind == 0 || kind == 1) {  // Ex (s x 2m): [cos | -sin] (kind 1: times w_q / s^2)
    M.assign((size_t)s * 2 * m, 0.f);
    for (int x = 0; x < s; ++x)
      for (int q = 0; q < m; ++q) {
        const double w = kind == 1 ? (q == 0 ? 1.0 : 2.0) * wscale : 1.0;
        M[(size_t)x * 2 * m + q] = (float)(w * std::cos(ang(x, q)));
        M[(size_t)x * 2 * m + m + q] = (float)(-w * std::sin(ang(x, q)));
      }
  } else if (kind == 2 || kind == 3) {  // EyA / EyB (4m x s)
    M.assign((size_t)4 * m * s, 0.f);
    for (int p = 0; p < 2 * m; ++p)
      for (int y = 0; y < s; ++y) {
        const double c = std::cos(ang(ky[p], y)), sn = std::sin(ang(ky[p], y));
        M[(size_t)p * s + y] = (float)(kind == 2 ? c : sn);
        M[(size_t)(2 * m + p) * s + y] = (float)(kind == 2 ? -sn : c);
      }
  } else if (kind == 4 || kind == 5) {  // EyIre / EyIim (s x 4m)
    M.assign((size_t)s * 4 * m, 0.f);
    for (int y = 0; y < s; ++y)
      for (int p = 0; p < 2 * m; ++p) {
        const double c = std::cos(ang(ky[p], y)), sn = std::sin(ang(ky[p], y));
        M[(size_t)y * 4 * m + p] = (float)(kind == 4 ? c : sn);
        M[(size_t)y * 4 * m + 2 * m + p] = (float)(kind == 4 ? -sn : c);
      }
  } else {  // WxI (kind 6: w_q / s^2) / WxI1 (kind 7: 1), 2m x s: rows q -> w cos, rows m+q -> -w sin
    M.assign((size_t)2 * m * s, 0.f);
    for (int q = 0; q < m; ++q)
      for (int x = 0; x < s; ++x) {
        const double w = kind == 6 ? (q == 0 ? 1.0 : 2.0) * wscale : 1.0;
        M[(size_t)q * s + x] = (float)(w * std::cos(ang(q, x)));
        M[(size_t)(m + q) * s + x] = (float)(-w * std::sin(ang(q, x)));
      }
  }
  return M;
}

}  // namespace

extern "C" {

sn_status sn_fno_create(sn_fno* out, int s, int c_in, int width, int modes, int layers, int proj,
                        int batch_max, void* cuda_stream) {
  if (!out) return ffail(SN_EINVAL, "sn_fno_create: out is NULL");
  *out = nullptr;
  if (s < 8 || c_in < 2 || width < 1 || modes < 1 || 2 * modes > s || layers < 1 || proj < 1 ||
      batch_max < 1)
    return ffail(SN_EINVAL, "sn_fno_create: need s >= 8, c_in >= 2, 1 <= 2 modes <= s, layers, "
                            "width, proj, batch_max >= 1");
  sn_fno f = new sn_fno_s();
  f->s = s; f->ci = c_in; f->C = width; f->m = modes; f->L = layers; f->J = proj; f->Bmax = batch_max;
  f->P = (ll)s * s;
  f->Nm = 2LL * modes * modes;
  auto bail = [&](sn_status st) { sn_fno_destroy(f); return st; };
  cudaError_t e;
  if (cuda_stream) {
    f->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else {
    if ((e = cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return bail(fcuda(e, "cudaStreamCreate"));
    f->own_stream = true;
  }
  // parameter layout (the oracle's order)
  ll off = 0;
  const ll C = width, Nm = f->Nm;
  f->off_P = off; off += C * c_in;
  f->off_pb = off; off += C;
  for (int l = 0; l < layers; ++l) {
    f->off_R.push_back(off); off += Nm * C * C * 2;
    f->off_W.push_back(off); off += C * C;
    f->off_b.push_back(off); off += C;
  }
  f->off_Q1 = off; off += (ll)proj * C;
  f->off_q1b = off; off += proj;
  f->off_Q2 = off; off += 3LL * proj;
  f->off_q2b = off; off += 3;
  f->nparams = off;
  const ll B = batch_max, P = f->P;
  if ((e = falloc(f, &f->params, off)) != cudaSuccess || (e = falloc(f, &f->grads, off)) != cudaSuccess ||
      (e = falloc(f, &f->am, off)) != cudaSuccess || (e = falloc(f, &f->av, off)) != cudaSuccess)
    return bail(fcuda(e, "cudaMalloc(params)"));
  cudaMemset(f->params, 0, off * sizeof(float));
  cudaMemset(f->am, 0, off * sizeof(float));
  cudaMemset(f->av, 0, off * sizeof(float));
  const int kinds[8] = {0, 1, 2, 3, 4, 5, 6, 7};
  float** mats[8] = {&f->ExF, &f->ExFw, &f->EyA, &f->EyB, &f->EyIre, &f->EyIim, &f->WxI, &f->WxI1};
  for (int k = 0; k < 8; ++k) {
    std::vector<float> M = dft_matrix(kinds[k], s, modes);
    if ((e = falloc(f, mats[k], M.size())) != cudaSuccess) return bail(fcuda(e, "cudaMalloc(dft)"));
    if ((e = cudaMemcpy(*mats[k], M.data(), M.size() * sizeof(float), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return bail(fcuda(e, "cudaMemcpy(dft)"));
  }
  const ll plane = B * C * P;
  f->v.assign(layers + 1, nullptr);
  f->z.assign(layers, nullptr);
  f->Vh.assign(layers, nullptr);
  bool ok = true;
  ok = ok && falloc(f, &f->a, B * c_in * P) == cudaSuccess;
  for (int l = 0; l <= layers; ++l) ok = ok && falloc(f, &f->v[l], plane) == cudaSuccess;
  for (int l = 0; l < layers; ++l) {
    ok = ok && falloc(f, &f->z[l], plane) == cudaSuccess;
    ok = ok && falloc(f, &f->Vh[l], B * C * 2 * Nm) == cudaSuccess;
  }
  ok = ok && falloc(f, &f->A1, B * C * s * 2LL * modes) == cudaSuccess;
  ok = ok && falloc(f, &f->B1, B * C * s * 2LL * modes) == cudaSuccess;
  ok = ok && cudaMalloc(&f->status, sizeof(int)) == cudaSuccess &&
       cudaMemset(f->status, 0, sizeof(int)) == cudaSuccess;
  ok = ok && falloc(f, &f->Uh, B * C * 2 * Nm) == cudaSuccess;
  ok = ok && falloc(f, &f->GU, B * C * 2 * Nm) == cudaSuccess;
  ok = ok && falloc(f, &f->GV, B * C * 2 * Nm) == cudaSuccess;
  ok = ok && falloc(f, &f->g1, B * proj * P) == cudaSuccess;
  ok = ok && falloc(f, &f->h, B * proj * P) == cudaSuccess;
  ok = ok && falloc(f, &f->dh, B * proj * P) == cudaSuccess;
  ok = ok && falloc(f, &f->out, B * 2 * P) == cudaSuccess;
  ok = ok && falloc(f, &f->yh, B * 3 * P) == cudaSuccess;
  ok = ok && falloc(f, &f->dy, B * 3 * P) == cudaSuccess;
  ok = ok && falloc(f, &f->dout, B * 2 * P) == cudaSuccess;
  ok = ok && falloc(f, &f->dv, plane) == cudaSuccess;
  ok = ok && falloc(f, &f->dv2, plane) == cudaSuccess;
  ok = ok && falloc(f, &f->dz, plane) == cudaSuccess;
  ok = ok && falloc(f, &f->norms, 3 * B) == cudaSuccess;
  ok = ok && falloc(f, &f->loss_part, 2 * B * kLossParts) == cudaSuccess;
  ok = ok && falloc(f, &f->chan_part, kChanParts * (size_t)std::max<ll>(proj, width)) == cudaSuccess;
  const ll nsplit = (P + kWgChunk - 1) / kWgChunk;
  const ll mn = std::max<ll>((ll)proj * C, std::max<ll>(C * C, C * (ll)c_in));
  f->work_floats = B * nsplit * std::max<ll>(mn, 3LL * proj);
  ok = ok && falloc(f, &f->work, f->work_floats) == cudaSuccess;
  {
    // per-mode mixing keeps V, GU (B x C) and R (C x C) of one mode in shared memory
    const size_t sm_fwd = sizeof(float2) * ((size_t)B * C + (size_t)C * C);
    const size_t sm_bwd = sizeof(float2) * (2 * (size_t)B * C + (size_t)C * (C + 1));
    if (sm_bwd > 200 * 1024) return bail(ffail(SN_ENOTSUP, "sn_fno_create: batch_max * width too large"));
    ok = ok && cudaFuncSetAttribute(mode_mix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sm_fwd) == cudaSuccess;
    if (mode_mix8_smem(B, C) <= 200 * 1024)
      ok = ok && cudaFuncSetAttribute(mode_mix8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)mode_mix8_smem(B, C)) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(mode_mix_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sm_bwd) == cudaSuccess;
  }
  {
    int dev = 0;
    ok = ok && cudaGetDevice(&dev) == cudaSuccess &&
         cudaDeviceGetAttribute(&f->sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
  }
  if (dfty_supported(s, modes)) {
    const int sm = (int)dfty_smem(s, modes);
    const size_t tn = (size_t)4 * modes * 2 * s;  // BF16 values of the table
    ok = ok && falloc(f, &f->EyAB, tn) == cudaSuccess;
    if (ok) {
      dfty_table_kernel<<<(unsigned)((tn + 255) / 256), 256, 0, f->stream>>>(f->EyA, f->EyB, f->EyAB, s,
                                                                             modes);
      ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(f->stream) == cudaSuccess;
    }
    ok = ok && cudaFuncSetAttribute(dft_y_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(dft_y_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(dft_y_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(dft_y_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
  }
  if (dfty_supported(s, modes)) {
    const int sm = (int)dftx_smem(s, modes);  // at most 2 x 32 x 264 BF16 values
    ok = ok && cudaFuncSetAttribute(dft_x_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(dft_x_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(dft_x_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(dft_x_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(dft_x_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(dft_x_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(dft_x_kernel<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(dft_x_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
  }
  if (dfty_supported(s, modes) && idfty_smem(s, modes) <= 200 * 1024) {
    const int sm = (int)idfty_smem(s, modes);
    const ll n = (ll)s * 4 * modes;  // values of EyIre (and of EyIim)
    ok = ok && falloc(f, &f->EyI, (size_t)(2 * n)) == cudaSuccess;
    if (ok) {
      stack_bf16_kernel<<<(unsigned)((2 * n + 255) / 256), 256, 0, f->stream>>>(f->EyIre, f->EyIim, f->EyI, n);
      ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(f->stream) == cudaSuccess;
    }
    ok = ok && cudaFuncSetAttribute(idft_y_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(idft_y_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(idft_y_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(idft_y_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) == cudaSuccess;
  }
  if (!ok) return bail(ffail(SN_ENOMEM, "sn_fno_create: device allocation failed"));
  if (fno_layer_umma_supported(f->C, 2 * f->m, f->s)) f->layer_form = SN_FNO_LAYER_UMMA;
  *out = f;
  return SN_OK;
}

long long sn_fno_param_count(sn_fno f) { return f ? f->nparams : 0; }

sn_status sn_fno_set_params(sn_fno f, const float* p, int on_device) {
  if (!f || !p) return ffail(SN_EINVAL, "sn_fno_set_params: NULL argument");
  FCHK(cudaMemcpyAsync(f->params, p, f->nparams * sizeof(float),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, f->stream));
  FCHK(cudaMemsetAsync(f->am, 0, f->nparams * sizeof(float), f->stream));
  FCHK(cudaMemsetAsync(f->av, 0, f->nparams * sizeof(float), f->stream));
  FCHK(cudaStreamSynchronize(f->stream));
  return SN_OK;
}

sn_status sn_fno_get_params(sn_fno f, float* p, int on_device) {
  if (!f || !p) return ffail(SN_EINVAL, "sn_fno_get_params: NULL argument");
  FCHK(cudaMemcpyAsync(p, f->params, f->nparams * sizeof(float),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, f->stream));
  FCHK(cudaStreamSynchronize(f->stream));
  return SN_OK;
}

sn_status sn_fno_get_grads(sn_fno f, float* g, int on_device) {
  if (!f || !g) return ffail(SN_EINVAL, "sn_fno_get_grads: NULL argument");
  FCHK(cudaMemcpyAsync(g, f->grads, f->nparams * sizeof(float),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, f->stream));
  FCHK(cudaStreamSynchronize(f->stream));
  return SN_OK;
}

sn_status sn_fno_set_grads(sn_fno f, const float* g, int on_device) {
  if (!f || !g) return ffail(SN_EINVAL, "sn_fno_set_grads: NULL argument");
  FCHK(cudaMemcpyAsync(f->grads, g, f->nparams * sizeof(float),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, f->stream));
  FCHK(cudaStreamSynchronize(f->stream));
  return SN_OK;
}

sn_status sn_fno_forward(sn_fno f, const float* in, float* out, int B) {
  if (!f || !in || !out) return ffail(SN_EINVAL, "sn_fno_forward: NULL argument");
  if (B < 1 || B > f->Bmax) return ffail(SN_EINVAL, "sn_fno_forward: batch must be in [1, batch_max]");
  const ll P = f->P, C = f->C, ci = f->ci, J = f->J;
  cudaStream_t st = f->stream;
  float* prm = f->params;
  FCHK(cudaMemcpyAsync(f->a, in, (size_t)B * ci * P * sizeof(float), cudaMemcpyDeviceToDevice, st));
  // lift: one pass over the input on the CUDA cores (few input channels)
  if (ci <= kLiftMaxIn && P % 4 == 0 && (C * ci + C) * sizeof(float) <= 48 * 1024) {
    lift_kernel<<<blocks_for(B * P / 4), 256, (size_t)(C * ci + C) * sizeof(float), st>>>(
        f->a, prm + f->off_P, prm + f->off_pb, f->v[0], (int)ci, (int)C, P, B);
  } else {
    FCHK(gemm(f, (int)C, (int)P, (int)ci, B, prm + f->off_P, 0, ci, 1, f->a, ci * P, P, 1, f->v[0], C * P, P, 1));
    bias_act_kernel<<<rows_grid(B * C, P), 256, 0, st>>>(f->v[0], prm + f->off_pb, nullptr, C, P, 0);
  }
  FCHK(cudaGetLastError());
  for (int l = 0; l < f->L; ++l) {
    FCHK(dft_forward(f, f->v[l], B, (int)C, f->ExF, f->Vh[l]));
    FCHK(mode_mix(f, f->Vh[l], prm + f->off_R[l], B, f->Uh));
    const int act = l < f->L - 1 ? 1 : 0;
    if (f->layer_form == SN_FNO_LAYER_UMMA) {
      // the inverse DFT along x, the 1x1 convolution, bias and activation in one kernel
      FCHK(dft_inverse_y(f, f->Uh, B, (int)C));
      FCHK(launch_fno_layer_umma(f->v[l], f->B1, f->WxI, prm + f->off_W[l], prm + f->off_b[l],
                                 f->z[l], f->v[l + 1], nullptr, B, (int)C, f->s, 2 * f->m, act, 0,
                                 f->status, st));
      continue;
    }
    FCHK(dft_inverse(f, f->Uh, B, (int)C, f->WxI, f->z[l], 0.f));
    // z = W v + the spectral branch + bias, and v' = GELU(z) (or z), in the GEMM's epilogue
    FCHK(gemm(f, (int)C, (int)P, (int)C, B, prm + f->off_W[l], 0, C, 1, f->v[l], C * P, P, 1, f->z[l],
              C * P, P, 1, 1.f, 1.f, prm + f->off_b[l], f->v[l + 1], act));
  }
  // projection
  // g1 = Q1 v + bias and h = GELU(g1) in the GEMM's epilogue
  FCHK(gemm(f, (int)J, (int)P, (int)C, B, prm + f->off_Q1, 0, C, 1, f->v[f->L], C * P, P, 1, f->g1,
            J * P, P, 1, 1.f, 0.f, prm + f->off_q1b, f->h, 1));
  if (P % 4 == 0 && 3 * J * sizeof(float) <= 48 * 1024) {
    // the last 1x1 (three outputs) and the head in one pass over h
    proj_head_kernel<<<blocks_for(B * P / 4), 256, (size_t)3 * J * sizeof(float), st>>>(
        f->h, prm + f->off_Q2, prm + f->off_q2b, f->a, f->yh, f->out, (int)J, (int)ci, P, B);
  } else {
    FCHK(gemm(f, 3, (int)P, (int)J, B, prm + f->off_Q2, 0, J, 1, f->h, J * P, P, 1, f->yh, 3 * P, P, 1));
    bias_act_kernel<<<rows_grid(B * 3, P), 256, 0, st>>>(f->yh, prm + f->off_q2b, nullptr, 3, P, 0);
    head_kernel<<<blocks_for(B * P), 256, 0, st>>>(f->a, f->yh, f->out, ci, P, B * P);
  }
  FCHK(cudaGetLastError());
  if (out != f->out)
    FCHK(cudaMemcpyAsync(out, f->out, (size_t)B * 2 * P * sizeof(float), cudaMemcpyDeviceToDevice, st));
  f->lastB = B;
  return SN_OK;
}

sn_status sn_fno_loss(sn_fno f, const float* target, int B, double* loss) {
  if (!f || !target || !loss) return ffail(SN_EINVAL, "sn_fno_loss: NULL argument");
  if (B != f->lastB) return ffail(SN_EINVAL, "sn_fno_loss: batch differs from the last forward");
  const ll n_per = 2 * f->P;
  loss_parts_kernel<<<dim3((unsigned)B, kLossParts), 256, 0, f->stream>>>(f->out, target, n_per,
                                                                           f->loss_part);
  loss_final_kernel<<<(unsigned)((B + 127) / 128), 128, 0, f->stream>>>(f->loss_part, B, f->norms);
  loss_grad_kernel<<<blocks_for(B * n_per), 256, 0, f->stream>>>(f->out, target, f->norms, n_per, B, f->dout);
  FCHK(cudaGetLastError());
  std::vector<double> nr(2 * B);
  FCHK(cudaMemcpyAsync(nr.data(), f->norms, nr.size() * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
  FCHK(cudaStreamSynchronize(f->stream));
  double s = 0.0;
  for (int b = 0; b < B; ++b) s += std::sqrt(nr[2 * b]) / std::sqrt(nr[2 * b + 1]);
  *loss = s / B;
  return SN_OK;
}

sn_status sn_fno_backward(sn_fno f) {
  if (!f || f->lastB < 1) return ffail(SN_EINVAL, "sn_fno_backward: no forward to differentiate");
  const int B = f->lastB;
  const ll P = f->P, C = f->C, ci = f->ci, J = f->J;
  cudaStream_t st = f->stream;
  float* prm = f->params;
  float* gr = f->grads;
  // head and projection
  head_bwd_kernel<<<blocks_for(B * P), 256, 0, st>>>(f->a, f->yh, f->dout, f->dy, ci, P, B * P);
  FCHK(cudaGetLastError());
  FCHK(weight_grad(f, f->dy, f->h, B, 3, (int)J, gr + f->off_Q2));
  channel_sum(f, f->dy, B, 3, P, gr + f->off_q2b);
  if (P % 4 == 0) {
    proj_dh_kernel<<<blocks_for(B * J * P / 4), 256, 0, st>>>(f->dy, prm + f->off_Q2, f->g1, f->dh,
                                                             (int)J, P, B);
  } else {
    FCHK(gemm(f, (int)J, (int)P, 3, B, prm + f->off_Q2, 0, 1, J, f->dy, 3 * P, P, 1, f->dh, J * P, P, 1));
    gelu_bwd_kernel<<<blocks_for(B * J * P), 256, 0, st>>>(f->dh, f->g1, f->dh, B * J * P);
  }
  FCHK(cudaGetLastError());
  FCHK(weight_grad(f, f->dh, f->v[f->L], B, (int)J, (int)C, gr + f->off_Q1));
  channel_sum(f, f->dh, B, J, P, gr + f->off_q1b);
  FCHK(gemm(f, (int)C, (int)P, (int)J, B, prm + f->off_Q1, 0, 1, C, f->dh, J * P, P, 1, f->dv, C * P, P, 1));
  if (f->layer_form == SN_FNO_LAYER_UMMA) {
    // dz of the last layer is dv (no activation after it); each layer's fused
    // kernel leaves the next one's dz: (W^T dz + the spectral branch) times
    // GELU' of the layer below, or, below layer 0, the lift's gradient dv
    float* dz = f->dv;
    float* nxt = f->dz;
    for (int l = f->L - 1; l >= 0; --l) {
      FCHK(weight_grad(f, dz, f->v[l], B, (int)C, (int)C, gr + f->off_W[l]));
      channel_sum(f, dz, B, C, P, gr + f->off_b[l]);
      FCHK(dft_forward(f, dz, B, (int)C, f->ExFw, f->GU));
      FCHK(mode_mix_bwd(f, f->Vh[l], prm + f->off_R[l], f->GU, B, gr + f->off_R[l], f->GV));
      FCHK(dft_inverse_y(f, f->GV, B, (int)C));
      FCHK(launch_fno_layer_umma(dz, f->B1, f->WxI1, prm + f->off_W[l], nullptr, nullptr, nxt,
                                 l > 0 ? f->z[l - 1] : nullptr, B, (int)C, f->s, 2 * f->m, 0, 1,
                                 f->status, st));
      std::swap(dz, nxt);
    }
    FCHK(weight_grad(f, dz, f->a, B, (int)C, (int)ci, gr + f->off_P));
    channel_sum(f, dz, B, C, P, gr + f->off_pb);
    FCHK(cudaGetLastError());
    return SN_OK;
  }
  for (int l = f->L - 1; l >= 0; --l) {
    const float* dz = f->dv;
    if (l < f->L - 1) {
      gelu_bwd_kernel<<<blocks_for(B * C * P), 256, 0, st>>>(f->dv, f->z[l], f->dz, B * C * P);
      FCHK(cudaGetLastError());
      dz = f->dz;
    }
    FCHK(weight_grad(f, dz, f->v[l], B, (int)C, (int)C, gr + f->off_W[l]));
    channel_sum(f, dz, B, C, P, gr + f->off_b[l]);
    FCHK(gemm(f, (int)C, (int)P, (int)C, B, prm + f->off_W[l], 0, 1, C, dz, C * P, P, 1, f->dv2, C * P, P, 1));
    // spectral branch
    FCHK(dft_forward(f, dz, B, (int)C, f->ExFw, f->GU));
    FCHK(mode_mix_bwd(f, f->Vh[l], prm + f->off_R[l], f->GU, B, gr + f->off_R[l], f->GV));
    FCHK(dft_inverse(f, f->GV, B, (int)C, f->WxI1, f->dv2, 1.f));
    std::swap(f->dv, f->dv2);
  }
  FCHK(weight_grad(f, f->dv, f->a, B, (int)C, (int)ci, gr + f->off_P));
  channel_sum(f, f->dv, B, C, P, gr + f->off_pb);
  FCHK(cudaGetLastError());
  return SN_OK;
}

sn_status sn_fno_adam(sn_fno f, double lr, double beta1, double beta2, double eps, int t) {
  if (!f || t < 1) return ffail(SN_EINVAL, "sn_fno_adam: bad argument");
  const float c1 = (float)(1.0 - std::pow(beta1, t)), c2 = (float)(1.0 - std::pow(beta2, t));
  adam_kernel<<<blocks_for(f->nparams), 256, 0, f->stream>>>(f->params, f->grads, f->am, f->av,
                                                               f->nparams, (float)lr, (float)beta1,
                                                               (float)beta2, (float)eps, c1, c2);
  FCHK(cudaGetLastError());
  return SN_OK;
}

sn_status sn_fno_sync(sn_fno f) {
  if (!f) return ffail(SN_EINVAL, "sn_fno_sync: NULL");
  FCHK(cudaStreamSynchronize(f->stream));
  int st = 0;
  FCHK(cudaMemcpy(&st, f->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    cudaMemset(f->status, 0, sizeof(int));
    return ffail(SN_ETIMEOUT, "sn_fno_sync: a bounded wait of the fused layer kernel expired");
  }
  return SN_OK;
}

sn_status sn_fno_set_layer_form(sn_fno f, int form) {
  if (!f) return ffail(SN_EINVAL, "sn_fno_set_layer_form: NULL");
  if (form != SN_FNO_LAYER_GEMMS && form != SN_FNO_LAYER_UMMA)
    return ffail(SN_EINVAL, "sn_fno_set_layer_form: unknown form");
  if (form == SN_FNO_LAYER_UMMA && !fno_layer_umma_supported(f->C, 2 * f->m, f->s))
    return ffail(SN_ENOTSUP, "sn_fno_set_layer_form: the fused layer takes width <= 64, 2 modes <= 64, "
                             "s <= 256");
  f->layer_form = form;
  return SN_OK;
}

void sn_fno_destroy(sn_fno f) {
  if (!f) return;
  if (f->stream) cudaStreamSynchronize(f->stream);
  if (f->status) cudaFree(f->status);
  for (void* p : f->allocs) cudaFree(p);
  if (f->own_stream && f->stream) cudaStreamDestroy(f->stream);
  delete f;
}

sn_status sn_fno_pack(const float* psi, const float* feats, int nfeat, float* X, int B,
                       long long cells, void* cuda_stream) {
  if (!psi || !X || B < 1 || cells < 1 || nfeat < 0 || (nfeat > 0 && !feats))
    return ffail(SN_EINVAL, "sn_fno_pack: bad argument");
  pack_kernel<<<blocks_for((ll)B * cells), 256, 0, (cudaStream_t)cuda_stream>>>(
      reinterpret_cast<const float2*>(psi), feats, nfeat, X, cells, (ll)B * cells);
  FCHK(cudaGetLastError());
  return SN_OK;
}

sn_status sn_fno_pack2(const float* psi_a, const float* psi_c, const float* feats, int nfeat,
                       float* X, int B, long long cells, void* cuda_stream) {
  if (!psi_a || !psi_c || !X || B < 1 || cells < 1 || nfeat < 0 || (nfeat > 0 && !feats))
    return ffail(SN_EINVAL, "sn_fno_pack2: bad argument");
  pack2_kernel<<<blocks_for((ll)B * cells), 256, 0, (cudaStream_t)cuda_stream>>>(
      reinterpret_cast<const float2*>(psi_a), reinterpret_cast<const float2*>(psi_c), feats, nfeat,
      X, cells, (ll)B * cells);
  FCHK(cudaGetLastError());
  return SN_OK;
}

sn_status sn_fno_unpack(const float* Y, float* psi, int B, long long cells, void* cuda_stream) {
  if (!Y || !psi || B < 1 || cells < 1) return ffail(SN_EINVAL, "sn_fno_unpack: bad argument");
  unpack_kernel<<<blocks_for((ll)B * cells), 256, 0, (cudaStream_t)cuda_stream>>>(
      Y, reinterpret_cast<float2*>(psi), cells, (ll)B * cells);
  FCHK(cudaGetLastError());
  return SN_OK;
}

sn_status sn_mass_c64(const float* psi, int B, long long cells, double* out, void* cuda_stream) {
  if (!psi || !out || B < 1 || cells < 1) return ffail(SN_EINVAL, "sn_mass_c64: bad argument");
  mass_kernel<<<B, 256, 0, (cudaStream_t)cuda_stream>>>(reinterpret_cast<const float2*>(psi), cells, out);
  FCHK(cudaGetLastError());
  return SN_OK;
}

sn_status sn_test_gemm_bf16(const float* A, long long sAz, long long sAm, long long sAk,
                            const float* B, long long sBz, long long sBk, long long sBn, float* C,
                            long long sCz, long long sCm, long long sCn, int M, int N, int K, int Z,
                            float alpha, float beta) {
  GemmArgs g{};
  g.A = A; g.sAz = sAz; g.sAm = sAm; g.sAk = sAk;
  g.B = B; g.sBz = sBz; g.sBk = sBk; g.sBn = sBn;
  g.C = C; g.sCz = sCz; g.sCm = sCm; g.sCn = sCn;
  g.M = M; g.N = N; g.K = K; g.Z = Z; g.alpha = alpha; g.beta = beta;
  cudaError_t e = gemm_bf16(g, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? SN_OK : fcuda(e, "sn_test_gemm_bf16");
}

}  // extern "C"
