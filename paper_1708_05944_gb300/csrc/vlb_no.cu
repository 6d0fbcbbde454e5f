// Learned warm start: a small 1D spectral neural operator over the normalised
// radius that maps (Kn, inner wall speed, R_out/R_in) to the steady profiles of
// n, u^phi, T and q^R.  The paper has no learned component; this is the
// production pattern built around the solver.  All arithmetic runs in the
// kernels of this file: BF16 tensor-core GEMMs (mma.sync m16n8k16, FP32
// accumulation, operands rounded to BF16 on load), FP32 element-wise kernels
// and an FP32 Adam update.  Architecture and parameter layout: see vlb.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/vlb.h"

namespace {

// ------------------------------------------------------------------ BF16 GEMM
// C[i][j] = alpha * sum_k A(i, k) B(k, j) + beta * C[i][j], batched; A(i, k) is
// A[i * a_r + k * a_c], B(k, j) is B[k * b_r + j * b_c], C row-major with ldc.
struct GemmArgs {
  int M, N, K;
  const float* A;
  long long a_r, a_c, sA;
  const float* B;
  long long b_r, b_c, sB;
  float* C;
  long long ldc, sC;
  float alpha, beta;
};

constexpr int GT_M = 64, GT_N = 64, GT_K = 16, G_THREADS = 128;

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat16 l = __float2bfloat16_rn(lo), h = __float2bfloat16_rn(hi);
  return (unsigned)__bfloat16_as_ushort(l) | ((unsigned)__bfloat16_as_ushort(h) << 16);
}

__global__ void __launch_bounds__(G_THREADS) gemm_bf16_kernel(const __grid_constant__ GemmArgs g) {
  // shared tiles in BF16: A as [m][k], B transposed as [n][k] (k contiguous for the fragments)
  __shared__ __nv_bfloat16 As[GT_M][GT_K + 8];
  __shared__ __nv_bfloat16 Bs[GT_N][GT_K + 8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.y * GT_M, n0 = blockIdx.x * GT_N, bz = blockIdx.z;
  const float* A = g.A + bz * g.sA;
  const float* B = g.B + bz * g.sB;
  float* C = g.C + bz * g.sC;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // 2 x 2 warps of 32 x 32
  const int gid = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  for (int k0 = 0; k0 < g.K; k0 += GT_K) {
    for (int e = tid; e < GT_M * GT_K; e += G_THREADS) {
      const int i = e / GT_K, k = e % GT_K;
      const int gi = m0 + i, gk = k0 + k;
      const float v = (gi < g.M && gk < g.K) ? A[gi * g.a_r + gk * g.a_c] : 0.f;
      As[i][k] = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < GT_N * GT_K; e += G_THREADS) {
      const int j = e / GT_K, k = e % GT_K;
      const int gj = n0 + j, gk = k0 + k;
      const float v = (gj < g.N && gk < g.K) ? B[gk * g.b_r + gj * g.b_c] : 0.f;
      Bs[j][k] = __float2bfloat16_rn(v);
    }
    __syncthreads();
    unsigned af[2][4], bfr[4][2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int r = wm + a * 16 + gid;
      af[a][0] = *reinterpret_cast<const unsigned*>(&As[r][2 * tig]);
      af[a][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][2 * tig]);
      af[a][2] = *reinterpret_cast<const unsigned*>(&As[r][2 * tig + 8]);
      af[a][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][2 * tig + 8]);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int cidx = wn + b * 8 + gid;
      bfr[b][0] = *reinterpret_cast<const unsigned*>(&Bs[cidx][2 * tig]);
      bfr[b][1] = *reinterpret_cast<const unsigned*>(&Bs[cidx][2 * tig + 8]);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(acc[a][b][0]), "+f"(acc[a][b][1]), "+f"(acc[a][b][2]), "+f"(acc[a][b][3])
            : "r"(af[a][0]), "r"(af[a][1]), "r"(af[a][2]), "r"(af[a][3]), "r"(bfr[b][0]), "r"(bfr[b][1]));
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = m0 + wm + a * 16 + gid + h * 8;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int j = n0 + wn + b * 8 + 2 * tig + q;
          if (i < g.M && j < g.N) {
            float* dst = C + i * g.ldc + j;
            const float v = g.alpha * acc[a][b][h * 2 + q];
            *dst = g.beta == 0.f ? v : v + g.beta * *dst;
          }
        }
      }
}

cudaError_t gemm(cudaStream_t s, int M, int N, int K, const float* A, long long a_r, long long a_c, long long sA,
                 const float* B, long long b_r, long long b_c, long long sB, float* C, long long ldc, long long sC,
                 int batch, float alpha = 1.f, float beta = 0.f) {
  GemmArgs g{M, N, K, A, a_r, a_c, sA, B, b_r, b_c, sB, C, ldc, sC, alpha, beta};
  dim3 grid((N + GT_N - 1) / GT_N, (M + GT_M - 1) / GT_M, batch);
  gemm_bf16_kernel<<<grid, G_THREADS, 0, s>>>(g);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ element-wise
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float dgelu_f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// features per grid point: [(log10 Kn + 1)/2, (u_w - 0.255)/0.245, (ratio - 2.75)/1.25, 2 s - 1]
__global__ void featurize_kernel(const float* cond, float* x, int B, int M) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B * M) return;
  const int b = r / M, m = r - b * M;
  x[4 * r + 0] = (log10f(cond[3 * b]) + 1.f) * 0.5f;
  x[4 * r + 1] = (cond[3 * b + 1] - 0.255f) / 0.245f;
  x[4 * r + 2] = (cond[3 * b + 2] - 2.75f) / 1.25f;
  x[4 * r + 3] = 2.f * (m + 0.5f) / M - 1.f;
}

// z += bias (rows x n); out = act(z) (act 0: identity, 1: GELU)
__global__ void bias_act_kernel(float* z, const float* bias, float* out, long long rows, int n, int act) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= rows * n) return;
  const float v = z[e] + bias[e % n];
  z[e] = v;
  if (out) out[e] = act ? gelu_f(v) : v;
}

__global__ void gelu_bwd_kernel(const float* dout, const float* pre, float* din, long long n) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < n) din[e] = dout[e] * dgelu_f(pre[e]);
}

// column sums of a (rows x n) matrix into out (n), one block per column
__global__ void colsum_kernel(const float* a, float* out, long long rows, int n) {
  __shared__ float red[256];
  const int j = blockIdx.x;
  float s = 0.f;
  for (long long r = threadIdx.x; r < rows; r += blockDim.x) s += a[r * n + j];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

// mean squared error and its gradient; loss accumulated in FP64
__global__ void mse_kernel(const float* y, const float* t, float* dy, long long n, double* loss) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float d = y[e] - t[e];
    dy[e] = 2.f * d / float(n);
    s += double(d) * double(d);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / double(n));
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gg = g[e];
  const float mm = b1 * m[e] + (1.f - b1) * gg;
  const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
  m[e] = mm;
  v[e] = vv;
  p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

inline int nblk(long long n, int t = 256) { return int((n + t - 1) / t); }

}  // namespace

struct vlb_no {
  int M, C, K, L, H;
  long long P;
  cudaStream_t stream = nullptr;
  float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
  long long adam_t = 0;
  float *D = nullptr, *Dinv = nullptr;
  std::vector<long long> off;  // parameter offsets: W_in, b_in, (S, W, b) x L, P1, c1, P2, c2
  int cap = 0;                 // batch capacity of the activation buffers
  float *cond = nullptr, *x = nullptr, *tgt = nullptr, *y = nullptr, *dy = nullptr;
  std::vector<float*> h, z, Hm;
  float *Om = nullptr, *s = nullptr, *a = nullptr, *ga = nullptr, *da = nullptr, *dh = nullptr, *dh2 = nullptr;
  float *dz = nullptr, *dOm = nullptr, *dHm = nullptr;
  double* loss = nullptr;
  float tmean[4] = {0, 0, 0, 0}, tstd[4] = {1, 1, 1, 1};
  std::string err;
};

namespace {

vlb_status no_fail(vlb_no* o, vlb_status s, const std::string& m) {
  if (o) o->err = m;
  return s;
}

#define NO_CUDA(o, call)                                                                  \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return no_fail((o), VLB_ERR_CUDA, std::string(#call) + ": " + \
                                                              cudaGetErrorString(e_));    \
  } while (0)

vlb_status ensure_capacity(vlb_no* o, int B) {
  if (B <= o->cap) return VLB_OK;
  auto fr = [](float*& p) {
    cudaFree(p);
    p = nullptr;
  };
  for (float*& p : o->h) fr(p);
  for (float*& p : o->z) fr(p);
  for (float*& p : o->Hm) fr(p);
  for (float** p : {&o->cond, &o->x, &o->tgt, &o->y, &o->dy, &o->Om, &o->s, &o->a, &o->ga, &o->da, &o->dh, &o->dh2,
                    &o->dz, &o->dOm, &o->dHm})
    fr(*p);
  const long long BM = (long long)B * o->M;
  auto al = [&](float*& p, long long n) { return cudaMalloc(&p, sizeof(float) * size_t(n)); };
  NO_CUDA(o, al(o->cond, 3LL * B));
  NO_CUDA(o, al(o->x, BM * 4));
  NO_CUDA(o, al(o->tgt, BM * 4));
  NO_CUDA(o, al(o->y, BM * 4));
  NO_CUDA(o, al(o->dy, BM * 4));
  o->h.assign(o->L + 1, nullptr);
  o->z.assign(o->L, nullptr);
  o->Hm.assign(o->L, nullptr);
  for (int l = 0; l <= o->L; ++l) NO_CUDA(o, al(o->h[l], BM * o->C));
  for (int l = 0; l < o->L; ++l) {
    NO_CUDA(o, al(o->z[l], BM * o->C));
    NO_CUDA(o, al(o->Hm[l], (long long)B * 2 * o->K * o->C));
  }
  NO_CUDA(o, al(o->Om, (long long)B * 2 * o->K * o->C));
  NO_CUDA(o, al(o->dOm, (long long)B * 2 * o->K * o->C));
  NO_CUDA(o, al(o->dHm, (long long)B * 2 * o->K * o->C));
  NO_CUDA(o, al(o->s, BM * o->C));
  NO_CUDA(o, al(o->dh, BM * o->C));
  NO_CUDA(o, al(o->dh2, BM * o->C));
  NO_CUDA(o, al(o->dz, BM * o->C));
  NO_CUDA(o, al(o->a, BM * o->H));
  NO_CUDA(o, al(o->ga, BM * o->H));
  NO_CUDA(o, al(o->da, BM * o->H));
  o->cap = B;
  return VLB_OK;
}

// forward pass for a batch whose conditions are already in o->cond
vlb_status forward(vlb_no* o, int B) {
  cudaStream_t st = o->stream;
  const int M = o->M, C = o->C, K = o->K, H = o->H;
  const long long BM = (long long)B * M;
  const float* p = o->params;
  featurize_kernel<<<nblk(BM), 256, 0, st>>>(o->cond, o->x, B, M);
  NO_CUDA(o, gemm(st, int(BM), C, 4, o->x, 4, 1, 0, p + o->off[0], C, 1, 0, o->h[0], C, 0, 1));
  bias_act_kernel<<<nblk(BM * C), 256, 0, st>>>(o->h[0], p + o->off[1], nullptr, BM, C, 0);
  for (int l = 0; l < o->L; ++l) {
    const float* S = p + o->off[2 + 3 * l];
    const float* W = p + o->off[3 + 3 * l];
    const float* bb = p + o->off[4 + 3 * l];
    // truncated DFT along the points: Hm[b] = D (2K x M) h[b] (M x C)
    NO_CUDA(o, gemm(st, 2 * K, C, M, o->D, M, 1, 0, o->h[l], C, 1, (long long)M * C, o->Hm[l], C,
                    (long long)2 * K * C, B));
    // per mode k: Om[:, k, :] (B x 2C) = Hm[:, k, :] (B x 2C) S[k] (2C x 2C)
    NO_CUDA(o, gemm(st, B, 2 * C, 2 * C, o->Hm[l], (long long)2 * K * C, 1, 2 * C, S, 2 * C, 1,
                    (long long)4 * C * C, o->Om, (long long)2 * K * C, 2 * C, K));
    // inverse truncated DFT: s[b] = Dinv (M x 2K) Om[b] (2K x C)
    NO_CUDA(o, gemm(st, M, C, 2 * K, o->Dinv, 2 * K, 1, 0, o->Om, C, 1, (long long)2 * K * C, o->z[l], C,
                    (long long)M * C, B));
    // z = s + h W + b, h_next = GELU(z) (identity on the last layer)
    NO_CUDA(o, gemm(st, int(BM), C, C, o->h[l], C, 1, 0, W, C, 1, 0, o->z[l], C, 0, 1, 1.f, 1.f));
    bias_act_kernel<<<nblk(BM * C), 256, 0, st>>>(o->z[l], bb, o->h[l + 1], BM, C, l < o->L - 1 ? 1 : 0);
  }
  const long long oP1 = o->off[2 + 3 * o->L];
  NO_CUDA(o, gemm(st, int(BM), H, C, o->h[o->L], C, 1, 0, p + oP1, H, 1, 0, o->a, H, 0, 1));
  bias_act_kernel<<<nblk(BM * H), 256, 0, st>>>(o->a, p + oP1 + (long long)C * H, o->ga, BM, H, 1);
  const long long oP2 = oP1 + (long long)C * H + H;
  NO_CUDA(o, gemm(st, int(BM), 4, H, o->ga, H, 1, 0, p + oP2, 4, 1, 0, o->y, 4, 0, 1));
  bias_act_kernel<<<nblk(BM * 4), 256, 0, st>>>(o->y, p + oP2 + (long long)H * 4, nullptr, BM, 4, 0);
  return cudaGetLastError() == cudaSuccess ? VLB_OK : no_fail(o, VLB_ERR_CUDA, "forward launch");
}

// loss and gradient into o->grads for the targets already in o->tgt (normalised)
vlb_status backward(vlb_no* o, int B) {
  cudaStream_t st = o->stream;
  const int M = o->M, C = o->C, K = o->K, H = o->H;
  const long long BM = (long long)B * M;
  const float* p = o->params;
  float* g = o->grads;
  NO_CUDA(o, cudaMemsetAsync(o->loss, 0, sizeof(double), st));
  mse_kernel<<<64, 256, 0, st>>>(o->y, o->tgt, o->dy, BM * 4, o->loss);
  const long long oP1 = o->off[2 + 3 * o->L], oP2 = oP1 + (long long)C * H + H;
  // y = ga P2 + c2
  NO_CUDA(o, gemm(st, H, 4, int(BM), o->ga, 1, H, 0, o->dy, 4, 1, 0, g + oP2, 4, 0, 1));
  colsum_kernel<<<4, 256, 0, st>>>(o->dy, g + oP2 + (long long)H * 4, BM, 4);
  NO_CUDA(o, gemm(st, int(BM), H, 4, o->dy, 4, 1, 0, p + oP2, 1, 4, 0, o->da, H, 0, 1));
  gelu_bwd_kernel<<<nblk(BM * H), 256, 0, st>>>(o->da, o->a, o->da, BM * H);
  // a = h_L P1 + c1
  NO_CUDA(o, gemm(st, C, H, int(BM), o->h[o->L], 1, C, 0, o->da, H, 1, 0, g + oP1, H, 0, 1));
  colsum_kernel<<<H, 256, 0, st>>>(o->da, g + oP1 + (long long)C * H, BM, H);
  NO_CUDA(o, gemm(st, int(BM), C, H, o->da, H, 1, 0, p + oP1, 1, H, 0, o->dh, C, 0, 1));
  for (int l = o->L - 1; l >= 0; --l) {
    const long long oS = o->off[2 + 3 * l], oW = o->off[3 + 3 * l], ob = o->off[4 + 3 * l];
    if (l < o->L - 1) gelu_bwd_kernel<<<nblk(BM * C), 256, 0, st>>>(o->dh, o->z[l], o->dz, BM * C);
    else NO_CUDA(o, cudaMemcpyAsync(o->dz, o->dh, sizeof(float) * BM * C, cudaMemcpyDeviceToDevice, st));
    NO_CUDA(o, gemm(st, C, C, int(BM), o->h[l], 1, C, 0, o->dz, C, 1, 0, g + oW, C, 0, 1));
    colsum_kernel<<<C, 256, 0, st>>>(o->dz, g + ob, BM, C);
    // dOm[b] = Dinv^T (2K x M) dz[b] (M x C)
    NO_CUDA(o, gemm(st, 2 * K, C, M, o->Dinv, 1, 2 * K, 0, o->dz, C, 1, (long long)M * C, o->dOm, C,
                    (long long)2 * K * C, B));
    // dS[k] = Hm[:, k, :]^T dOm[:, k, :]
    NO_CUDA(o, gemm(st, 2 * C, 2 * C, B, o->Hm[l], 1, (long long)2 * K * C, 2 * C, o->dOm, (long long)2 * K * C, 1,
                    2 * C, g + oS, 2 * C, (long long)4 * C * C, K));
    // dHm[:, k, :] = dOm[:, k, :] S[k]^T
    NO_CUDA(o, gemm(st, B, 2 * C, 2 * C, o->dOm, (long long)2 * K * C, 1, 2 * C, p + oS, 1, 2 * C,
                    (long long)4 * C * C, o->dHm, (long long)2 * K * C, 2 * C, K));
    // dh = dz W^T + D^T dHm[b]
    NO_CUDA(o, gemm(st, int(BM), C, C, o->dz, C, 1, 0, p + oW, 1, C, 0, o->dh2, C, 0, 1));
    NO_CUDA(o, gemm(st, M, C, 2 * K, o->D, 1, M, 0, o->dHm, C, 1, (long long)2 * K * C, o->dh2, C, (long long)M * C,
                    B, 1.f, 1.f));
    std::swap(o->dh, o->dh2);
  }
  NO_CUDA(o, gemm(st, 4, C, int(BM), o->x, 1, 4, 0, o->dh, C, 1, 0, g + o->off[0], C, 0, 1));
  colsum_kernel<<<C, 256, 0, st>>>(o->dh, g + o->off[1], BM, C);
  return cudaGetLastError() == cudaSuccess ? VLB_OK : no_fail(o, VLB_ERR_CUDA, "backward launch");
}

vlb_status upload_batch(vlb_no* o, const double* cond, const double* targets, int B) {
  vlb_status s = ensure_capacity(o, B);
  if (s != VLB_OK) return s;
  std::vector<float> c(3 * size_t(B));
  for (int i = 0; i < 3 * B; ++i) c[i] = float(cond[i]);
  for (int b = 0; b < B; ++b)
    if (!(cond[3 * b] > 0.0)) return no_fail(o, VLB_ERR_INVALID, "Kn must be positive");
  NO_CUDA(o, cudaMemcpyAsync(o->cond, c.data(), sizeof(float) * c.size(), cudaMemcpyHostToDevice, o->stream));
  if (targets) {
    const size_t n = size_t(B) * o->M * 4;
    std::vector<float> t(n);
    for (size_t e = 0; e < n; ++e) t[e] = float((targets[e] - o->tmean[e % 4]) / o->tstd[e % 4]);
    NO_CUDA(o, cudaMemcpyAsync(o->tgt, t.data(), sizeof(float) * n, cudaMemcpyHostToDevice, o->stream));
    NO_CUDA(o, cudaStreamSynchronize(o->stream));
  } else {
    NO_CUDA(o, cudaStreamSynchronize(o->stream));
  }
  return VLB_OK;
}

}  // namespace

extern "C" {

vlb_status vlb_no_create(int grid_points, int width, int modes, int layers, int hidden, void* cuda_stream,
                         vlb_no** out) {
  if (!out) return VLB_ERR_INVALID;
  *out = nullptr;
  if (grid_points < 4 || width < 1 || modes < 1 || 2 * modes > grid_points || layers < 1 || hidden < 1)
    return VLB_ERR_INVALID;
  vlb_no* o = new vlb_no;
  o->M = grid_points, o->C = width, o->K = modes, o->L = layers, o->H = hidden;
  o->stream = static_cast<cudaStream_t>(cuda_stream);
  long long n = 0;
  auto push = [&](long long sz) {
    o->off.push_back(n);
    n += sz;
  };
  push(4LL * width);
  push(width);
  for (int l = 0; l < layers; ++l) {
    push((long long)modes * 4 * width * width);
    push((long long)width * width);
    push(width);
  }
  push((long long)width * hidden);  // P1 (c1 follows it)
  n += hidden;
  push((long long)hidden * 4);  // P2 (c2 follows it)
  n += 4;
  o->P = n;
  auto bad = [&](cudaError_t e) {
    if (e == cudaSuccess) return false;
    o->err = cudaGetErrorString(e);
    return true;
  };
  if (bad(cudaMalloc(&o->params, sizeof(float) * n)) || bad(cudaMalloc(&o->grads, sizeof(float) * n)) ||
      bad(cudaMalloc(&o->am, sizeof(float) * n)) || bad(cudaMalloc(&o->av, sizeof(float) * n)) ||
      bad(cudaMalloc(&o->D, sizeof(float) * 2 * modes * grid_points)) ||
      bad(cudaMalloc(&o->Dinv, sizeof(float) * 2 * modes * grid_points)) || bad(cudaMalloc(&o->loss, sizeof(double)))) {
    vlb_no_destroy(o);
    return VLB_ERR_CUDA;
  }
  // DFT matrices, rows / columns ordered (mode, Re/Im)
  std::vector<float> D(2 * size_t(modes) * grid_points), Di(2 * size_t(modes) * grid_points);
  for (int k = 0; k < modes; ++k)
    for (int m = 0; m < grid_points; ++m) {
      const double th = 2.0 * M_PI * k * m / grid_points, ck = k == 0 ? 1.0 : 2.0;
      D[(2 * k) * grid_points + m] = float(cos(th));
      D[(2 * k + 1) * grid_points + m] = float(-sin(th));
      Di[m * 2 * modes + 2 * k] = float(ck * cos(th) / grid_points);
      Di[m * 2 * modes + 2 * k + 1] = float(-ck * sin(th) / grid_points);
    }
  cudaMemcpy(o->D, D.data(), sizeof(float) * D.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(o->Dinv, Di.data(), sizeof(float) * Di.size(), cudaMemcpyHostToDevice);
  cudaMemset(o->params, 0, sizeof(float) * n);
  cudaMemset(o->am, 0, sizeof(float) * n);
  cudaMemset(o->av, 0, sizeof(float) * n);
  *out = o;
  return VLB_OK;
}

long long vlb_no_num_params(const vlb_no* o) { return o ? o->P : -1; }

vlb_status vlb_no_set_params(vlb_no* o, const float* theta) {
  if (!o || !theta) return VLB_ERR_INVALID;
  NO_CUDA(o, cudaMemcpy(o->params, theta, sizeof(float) * o->P, cudaMemcpyHostToDevice));
  NO_CUDA(o, cudaMemset(o->am, 0, sizeof(float) * o->P));
  NO_CUDA(o, cudaMemset(o->av, 0, sizeof(float) * o->P));
  o->adam_t = 0;
  return VLB_OK;
}

vlb_status vlb_no_get_params(vlb_no* o, float* theta) {
  if (!o || !theta) return VLB_ERR_INVALID;
  NO_CUDA(o, cudaStreamSynchronize(o->stream));
  NO_CUDA(o, cudaMemcpy(theta, o->params, sizeof(float) * o->P, cudaMemcpyDeviceToHost));
  return VLB_OK;
}

vlb_status vlb_no_set_target_scaling(vlb_no* o, const double* mean, const double* std) {
  if (!o || !mean || !std) return VLB_ERR_INVALID;
  for (int c = 0; c < 4; ++c) {
    if (!(std[c] > 0.0)) return no_fail(o, VLB_ERR_INVALID, "scales must be positive");
    o->tmean[c] = float(mean[c]);
    o->tstd[c] = float(std[c]);
  }
  return VLB_OK;
}

vlb_status vlb_no_predict(vlb_no* o, const double* cond, int B, double* out) {
  if (!o || !cond || !out || B < 1) return VLB_ERR_INVALID;
  vlb_status s = upload_batch(o, cond, nullptr, B);
  if (s != VLB_OK) return s;
  s = forward(o, B);
  if (s != VLB_OK) return s;
  const size_t n = size_t(B) * o->M * 4;
  std::vector<float> y(n);
  NO_CUDA(o, cudaMemcpyAsync(y.data(), o->y, sizeof(float) * n, cudaMemcpyDeviceToHost, o->stream));
  NO_CUDA(o, cudaStreamSynchronize(o->stream));
  for (size_t e = 0; e < n; ++e) out[e] = double(y[e]) * o->tstd[e % 4] + o->tmean[e % 4];
  return VLB_OK;
}

vlb_status vlb_no_loss_and_grad(vlb_no* o, const double* cond, const double* targets, int B, double* loss,
                                float* grad) {
  if (!o || !cond || !targets || B < 1) return VLB_ERR_INVALID;
  vlb_status s = upload_batch(o, cond, targets, B);
  if (s == VLB_OK) s = forward(o, B);
  if (s == VLB_OK) s = backward(o, B);
  if (s != VLB_OK) return s;
  if (loss) NO_CUDA(o, cudaMemcpyAsync(loss, o->loss, sizeof(double), cudaMemcpyDeviceToHost, o->stream));
  if (grad) NO_CUDA(o, cudaMemcpyAsync(grad, o->grads, sizeof(float) * o->P, cudaMemcpyDeviceToHost, o->stream));
  NO_CUDA(o, cudaStreamSynchronize(o->stream));
  return VLB_OK;
}

vlb_status vlb_no_train_step(vlb_no* o, const double* cond, const double* targets, int B, double lr, double* loss) {
  if (!o || !cond || !targets || B < 1 || !(lr > 0.0)) return VLB_ERR_INVALID;
  vlb_status s = upload_batch(o, cond, targets, B);
  if (s == VLB_OK) s = forward(o, B);
  if (s == VLB_OK) s = backward(o, B);
  if (s != VLB_OK) return s;
  o->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, float(o->adam_t)), c2 = 1.f - powf(b2, float(o->adam_t));
  adam_kernel<<<nblk(o->P), 256, 0, o->stream>>>(o->params, o->grads, o->am, o->av, o->P, float(lr), b1, b2, 1e-8f,
                                                 c1, c2);
  if (loss) NO_CUDA(o, cudaMemcpyAsync(loss, o->loss, sizeof(double), cudaMemcpyDeviceToHost, o->stream));
  NO_CUDA(o, cudaStreamSynchronize(o->stream));
  return VLB_OK;
}

const char* vlb_no_last_error(const vlb_no* o) { return o ? o->err.c_str() : ""; }

void vlb_no_destroy(vlb_no* o) {
  if (!o) return;
  if (o->stream) cudaStreamSynchronize(o->stream);
  for (float* p : o->h) cudaFree(p);
  for (float* p : o->z) cudaFree(p);
  for (float* p : o->Hm) cudaFree(p);
  for (float* p : {o->params, o->grads, o->am, o->av, o->D, o->Dinv, o->cond, o->x, o->tgt, o->y, o->dy, o->Om, o->s,
                   o->a, o->ga, o->da, o->dh, o->dh2, o->dz, o->dOm, o->dHm})
    cudaFree(p);
  cudaFree(o->loss);
  delete o;
}

}  // extern "C"
