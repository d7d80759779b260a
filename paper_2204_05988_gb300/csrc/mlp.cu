// BF16 multilayer perceptron for the learned warm start (training and inference).
//
// y = W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3 per sample (row-major batches:
// X [B][n_in], H [B][w], Y [B][n_out]; W_k stored [fan_in][fan_out]).  GEMM
// operands are BF16 on the tensor cores (warp-level 16x16x16 fragments, FP32
// accumulation); master weights, biases, gradients and Adam moments are FP32.
// Loss: 1/(2B) sum (y - t)^2.  Inputs and targets enter and leave as FP64 and
// are scaled by in_scale / out_scale inside the kernels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sgdg.h"

namespace sgdg {

namespace {

using bf16 = __nv_bfloat16;
namespace wm = nvcuda::wmma;

constexpr int kT = 16;   // fragment edge

// C[M][N] (+)= sum_k A(m,k) B(k,n); A is [M][K] (TA = false) or [K][M] (TA = true),
// B is [K][N] (TB = false) or [N][K] (TB = true); all dims multiples of 16.
// One warp per 16x16 tile of C, 4 warps per block.
template <bool TA, bool TB>
__global__ void k_gemm(const bf16* A, const bf16* B, float* C, int M, int N, int K, int accumulate) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int tiles_n = N / kT;
  const int tm = warp / tiles_n, tn = warp % tiles_n;
  if (tm * kT >= M) return;
  using LA = typename std::conditional<TA, wm::col_major, wm::row_major>::type;
  using LB = typename std::conditional<TB, wm::col_major, wm::row_major>::type;
  wm::fragment<wm::matrix_a, kT, kT, kT, bf16, LA> fa;
  wm::fragment<wm::matrix_b, kT, kT, kT, bf16, LB> fb;
  wm::fragment<wm::accumulator, kT, kT, kT, float> fc;
  float* c = C + (size_t)tm * kT * N + tn * kT;
  if (accumulate) wm::load_matrix_sync(fc, c, N, wm::mem_row_major);
  else wm::fill_fragment(fc, 0.0f);
  for (int k = 0; k < K; k += kT) {
    const bf16* a = TA ? A + (size_t)k * M + tm * kT : A + (size_t)tm * kT * K + k;
    const bf16* b = TB ? B + (size_t)tn * kT * K + k : B + (size_t)k * N + tn * kT;
    wm::load_matrix_sync(fa, a, TA ? M : K);
    wm::load_matrix_sync(fb, b, TB ? K : N);
    wm::mma_sync(fc, fa, fb, fc);
  }
  wm::store_matrix_sync(c, fc, N, wm::mem_row_major);
}

template <bool TA, bool TB>
cudaError_t gemm(const bf16* A, const bf16* B, float* C, int M, int N, int K, int acc, cudaStream_t s) {
  const long long tiles = (long long)(M / kT) * (N / kT);
  const int threads = 128;
  const long long blocks = (tiles * 32 + threads - 1) / threads;
  k_gemm<TA, TB><<<(unsigned)blocks, threads, 0, s>>>(A, B, C, M, N, K, acc);
  return cudaGetLastError();
}

__global__ void k_to_bf16(const float* x, bf16* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}
// X [Bp][n] from FP64 rows (rows >= B zero), scaled
__global__ void k_load_rows(const double* x, int B, int Bp, int n, double scale, bf16* y) {
  long long tot = (long long)Bp * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    int b = (int)(i / n);
    y[i] = __float2bfloat16(b < B ? (float)(x[i] * scale) : 0.0f);
  }
}
// H = relu(Z + bias) -> bf16 copy and mask
__global__ void k_bias_relu(const float* Z, const float* bias, int Bp, int n, bf16* H, float* Hf) {
  long long tot = (long long)Bp * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    float z = Z[i] + bias[i % n];
    float h = z > 0.0f ? z : 0.0f;
    Hf[i] = h;
    H[i] = __float2bfloat16(h);
  }
}
// Y = Z + b, written as FP64 / out_scale for the first B rows
__global__ void k_bias_out(const float* Z, const float* bias, int B, int n, double inv_scale, double* y) {
  long long tot = (long long)B * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)(Z[i] + bias[i % n]) * inv_scale;
}
// dY = (Z + b - t * out_scale) / B (rows < B), 0 for padding rows; loss partial sums
__global__ void k_dloss(const float* Z, const float* bias, const double* t, int B, int Bp, int n, double out_scale,
                        float* dY, bf16* dYb, double* loss) {
  long long tot = (long long)Bp * n;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    int b = (int)(i / n);
    float g = 0.0f;
    if (b < B) {
      float r = Z[i] + bias[i % n] - (float)(t[i] * out_scale);
      acc += 0.5 * (double)r * r;
      g = r / (float)B;
    }
    dY[i] = g;
    dYb[i] = __float2bfloat16(g);
  }
  atomicAdd(loss, acc / B);
}
// dH = dHin * (H > 0) -> bf16
__global__ void k_relu_back(const float* dH, const float* H, long long n, bf16* dHb, float* dHf) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float g = H[i] > 0.0f ? dH[i] : 0.0f;
    dHf[i] = g;
    dHb[i] = __float2bfloat16(g);
  }
}
// db[j] = sum_b dY[b][j]
__global__ void k_colsum(const float* dY, int Bp, int n, float* db) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float s = 0.0f;
  for (int b = 0; b < Bp; ++b) s += dY[(size_t)b * n + j];
  db[j] = s;
}
__global__ void k_adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

int gsz(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }

struct Layer {
  int fin = 0, fout = 0;
  float *W = nullptr, *b = nullptr, *gW = nullptr, *gb = nullptr;
  float *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr;
  bf16* Wb = nullptr;
};

}  // namespace

struct Mlp {
  int n_in = 0, w = 0, n_out = 0, Bmax = 0;
  double in_scale = 1.0, out_scale = 1.0;
  Layer l[3];
  long long step = 0;
  // activations for the largest batch (padded to 16)
  bf16 *X = nullptr, *H1b = nullptr, *H2b = nullptr, *dYb = nullptr, *dH2b = nullptr, *dH1b = nullptr;
  float *Z = nullptr, *H1 = nullptr, *H2 = nullptr, *dY = nullptr, *dH = nullptr, *dHf = nullptr;
  double* loss = nullptr;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

cudaError_t mlp_alloc(Mlp& m, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) {
    m.allocs.push_back(*p);
    cudaMemset(*p, 0, bytes);
  }
  return e;
}

// splitmix64 -> uniform in [-1, 1)
double uniform_pm1(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

sgdg_status forward(Mlp& m, int B, int Bp, cudaStream_t s) {
  // layer 1
  if (gemm<false, false>(m.X, m.l[0].Wb, m.Z, Bp, m.w, m.n_in, 0, s) != cudaSuccess) return SGDG_ECUDA;
  k_bias_relu<<<gsz((long long)Bp * m.w), 256, 0, s>>>(m.Z, m.l[0].b, Bp, m.w, m.H1b, m.H1);
  if (gemm<false, false>(m.H1b, m.l[1].Wb, m.Z, Bp, m.w, m.w, 0, s) != cudaSuccess) return SGDG_ECUDA;
  k_bias_relu<<<gsz((long long)Bp * m.w), 256, 0, s>>>(m.Z, m.l[1].b, Bp, m.w, m.H2b, m.H2);
  if (gemm<false, false>(m.H2b, m.l[2].Wb, m.Z, Bp, m.n_out, m.w, 0, s) != cudaSuccess) return SGDG_ECUDA;
  return cudaGetLastError() == cudaSuccess ? SGDG_OK : SGDG_ECUDA;
}

void refresh_bf16(Mlp& m, cudaStream_t s) {
  for (auto& L : m.l) {
    long long n = (long long)L.fin * L.fout;
    k_to_bf16<<<gsz(n), 256, 0, s>>>(L.W, L.Wb, n);
  }
}

// gradients of the loss into l[k].gW / gb; loss into m.loss
sgdg_status backward(Mlp& m, const double* t, int B, int Bp, cudaStream_t s) {
  cudaMemsetAsync(m.loss, 0, sizeof(double), s);
  k_dloss<<<gsz((long long)Bp * m.n_out), 256, 0, s>>>(m.Z, m.l[2].b, t, B, Bp, m.n_out, m.out_scale, m.dY,
                                                         m.dYb, m.loss);
  // layer 3: gW3 = H2^T dY, gb3 = colsum dY, dH2 = dY W3^T
  if (gemm<true, false>(m.H2b, m.dYb, m.l[2].gW, m.w, m.n_out, Bp, 0, s) != cudaSuccess) return SGDG_ECUDA;
  k_colsum<<<(m.n_out + 255) / 256, 256, 0, s>>>(m.dY, Bp, m.n_out, m.l[2].gb);
  if (gemm<false, true>(m.dYb, m.l[2].Wb, m.dH, Bp, m.w, m.n_out, 0, s) != cudaSuccess) return SGDG_ECUDA;
  k_relu_back<<<gsz((long long)Bp * m.w), 256, 0, s>>>(m.dH, m.H2, (long long)Bp * m.w, m.dH2b, m.dHf);
  // layer 2
  if (gemm<true, false>(m.H1b, m.dH2b, m.l[1].gW, m.w, m.w, Bp, 0, s) != cudaSuccess) return SGDG_ECUDA;
  k_colsum<<<(m.w + 255) / 256, 256, 0, s>>>(m.dHf, Bp, m.w, m.l[1].gb);
  if (gemm<false, true>(m.dH2b, m.l[1].Wb, m.dH, Bp, m.w, m.w, 0, s) != cudaSuccess) return SGDG_ECUDA;
  k_relu_back<<<gsz((long long)Bp * m.w), 256, 0, s>>>(m.dH, m.H1, (long long)Bp * m.w, m.dH1b, m.dHf);
  // layer 1
  if (gemm<true, false>(m.X, m.dH1b, m.l[0].gW, m.n_in, m.w, Bp, 0, s) != cudaSuccess) return SGDG_ECUDA;
  k_colsum<<<(m.w + 255) / 256, 256, 0, s>>>(m.dHf, Bp, m.w, m.l[0].gb);
  return cudaGetLastError() == cudaSuccess ? SGDG_OK : SGDG_ECUDA;
}

sgdg_status load_batch(Mlp& m, const double* x, int B, int* Bp, cudaStream_t s) {
  if (B < 1 || B > m.Bmax) {
    m.err = "batch size out of range 1.." + std::to_string(m.Bmax);
    return SGDG_EINVAL;
  }
  *Bp = (B + kT - 1) / kT * kT;
  k_load_rows<<<gsz((long long)*Bp * m.n_in), 256, 0, s>>>(x, B, *Bp, m.n_in, m.in_scale, m.X);
  return cudaGetLastError() == cudaSuccess ? SGDG_OK : SGDG_ECUDA;
}

}  // namespace

}  // namespace sgdg

using namespace sgdg;

extern "C" {

sgdg_status sgdg_mlp_create(int n_in, int width, int n_out, int max_batch, unsigned long long seed, void** out) {
  if (!out || n_in <= 0 || width <= 0 || n_out <= 0 || max_batch <= 0 || n_in % 16 || width % 16 || n_out % 16)
    return SGDG_EINVAL;
  Mlp* m = new Mlp();
  m->n_in = n_in;
  m->w = width;
  m->n_out = n_out;
  m->Bmax = max_batch;
  const int dims[4] = {n_in, width, width, n_out};
  uint64_t st = seed;
  for (int k = 0; k < 3; ++k) {
    Layer& L = m->l[k];
    L.fin = dims[k];
    L.fout = dims[k + 1];
    const size_t nw = (size_t)L.fin * L.fout;
    if (mlp_alloc(*m, (void**)&L.W, 4 * nw) || mlp_alloc(*m, (void**)&L.gW, 4 * nw) ||
        mlp_alloc(*m, (void**)&L.mW, 4 * nw) || mlp_alloc(*m, (void**)&L.vW, 4 * nw) ||
        mlp_alloc(*m, (void**)&L.Wb, 2 * nw) || mlp_alloc(*m, (void**)&L.b, 4 * L.fout) ||
        mlp_alloc(*m, (void**)&L.gb, 4 * L.fout) || mlp_alloc(*m, (void**)&L.mb, 4 * L.fout) ||
        mlp_alloc(*m, (void**)&L.vb, 4 * L.fout)) {
      sgdg_mlp_destroy(m);
      return SGDG_ENOMEM;
    }
    // He-uniform initialisation (last layer scaled down), biases zero
    std::vector<float> w(nw);
    const double a = std::sqrt(6.0 / L.fin) * (k == 2 ? 0.1 : 1.0);
    for (auto& x : w) x = (float)(a * uniform_pm1(st));
    cudaMemcpy(L.W, w.data(), 4 * nw, cudaMemcpyHostToDevice);
  }
  const int Bp = (max_batch + 15) / 16 * 16;
  const int wide = std::max(width, n_out);
  if (mlp_alloc(*m, (void**)&m->X, 2ull * Bp * n_in) || mlp_alloc(*m, (void**)&m->H1b, 2ull * Bp * width) ||
      mlp_alloc(*m, (void**)&m->H2b, 2ull * Bp * width) || mlp_alloc(*m, (void**)&m->dYb, 2ull * Bp * n_out) ||
      mlp_alloc(*m, (void**)&m->dH2b, 2ull * Bp * width) || mlp_alloc(*m, (void**)&m->dH1b, 2ull * Bp * width) ||
      mlp_alloc(*m, (void**)&m->Z, 4ull * Bp * wide) || mlp_alloc(*m, (void**)&m->H1, 4ull * Bp * width) ||
      mlp_alloc(*m, (void**)&m->H2, 4ull * Bp * width) || mlp_alloc(*m, (void**)&m->dY, 4ull * Bp * n_out) ||
      mlp_alloc(*m, (void**)&m->dH, 4ull * Bp * width) || mlp_alloc(*m, (void**)&m->dHf, 4ull * Bp * width) ||
      mlp_alloc(*m, (void**)&m->loss, sizeof(double))) {
    sgdg_mlp_destroy(m);
    return SGDG_ENOMEM;
  }
  refresh_bf16(*m, nullptr);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    sgdg_mlp_destroy(m);
    return SGDG_ECUDA;
  }
  *out = m;
  return SGDG_OK;
}

void sgdg_mlp_destroy(void* p) {
  if (!p) return;
  Mlp* m = (Mlp*)p;
  cudaDeviceSynchronize();
  for (void* a : m->allocs) cudaFree(a);
  delete m;
}

sgdg_status sgdg_mlp_set_scaling(void* p, double in_scale, double out_scale) {
  if (!p || !(in_scale > 0.0) || !(out_scale > 0.0)) return SGDG_EINVAL;
  Mlp* m = (Mlp*)p;
  m->in_scale = in_scale;
  m->out_scale = out_scale;
  return SGDG_OK;
}

sgdg_status sgdg_mlp_forward(void* p, const double* x, int batch, double* y, void* stream) {
  if (!p || !x || !y) return SGDG_EINVAL;
  Mlp& m = *(Mlp*)p;
  cudaStream_t s = (cudaStream_t)stream;
  int Bp;
  sgdg_status st = load_batch(m, x, batch, &Bp, s);
  if (st) return st;
  st = forward(m, batch, Bp, s);
  if (st) return st;
  k_bias_out<<<gsz((long long)batch * m.n_out), 256, 0, s>>>(m.Z, m.l[2].b, batch, m.n_out, 1.0 / m.out_scale, y);
  return cudaGetLastError() == cudaSuccess ? SGDG_OK : SGDG_ECUDA;
}

sgdg_status sgdg_mlp_train_step(void* p, const double* x, const double* t, int batch, double lr, double* loss,
                                void* stream) {
  if (!p || !x || !t) return SGDG_EINVAL;
  Mlp& m = *(Mlp*)p;
  cudaStream_t s = (cudaStream_t)stream;
  int Bp;
  sgdg_status st = load_batch(m, x, batch, &Bp, s);
  if (st) return st;
  if ((st = forward(m, batch, Bp, s))) return st;
  if ((st = backward(m, t, batch, Bp, s))) return st;
  m.step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)m.step), c2 = 1.0f - powf(b2, (float)m.step);
  for (auto& L : m.l) {
    const long long nw = (long long)L.fin * L.fout;
    k_adam<<<gsz(nw), 256, 0, s>>>(L.W, L.gW, L.mW, L.vW, nw, (float)lr, b1, b2, c1, c2, 1e-8f);
    k_adam<<<gsz(L.fout), 256, 0, s>>>(L.b, L.gb, L.mb, L.vb, L.fout, (float)lr, b1, b2, c1, c2, 1e-8f);
  }
  refresh_bf16(m, s);
  if (loss) {
    if (cudaMemcpyAsync(loss, m.loss, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SGDG_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SGDG_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? SGDG_OK : SGDG_ECUDA;
}

sgdg_status sgdg_mlp_gradients(void* p, const double* x, const double* t, int batch, float* grads_host,
                               double* loss) {
  if (!p || !x || !t || !grads_host) return SGDG_EINVAL;
  Mlp& m = *(Mlp*)p;
  int Bp;
  sgdg_status st = load_batch(m, x, batch, &Bp, nullptr);
  if (st) return st;
  if ((st = forward(m, batch, Bp, nullptr))) return st;
  if ((st = backward(m, t, batch, Bp, nullptr))) return st;
  size_t o = 0;
  for (auto& L : m.l) {
    const size_t nw = (size_t)L.fin * L.fout;
    if (cudaMemcpy(grads_host + o, L.gW, 4 * nw, cudaMemcpyDeviceToHost) != cudaSuccess) return SGDG_ECUDA;
    o += nw;
    if (cudaMemcpy(grads_host + o, L.gb, 4 * L.fout, cudaMemcpyDeviceToHost) != cudaSuccess) return SGDG_ECUDA;
    o += L.fout;
  }
  if (loss && cudaMemcpy(loss, m.loss, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return SGDG_ECUDA;
  return SGDG_OK;
}

long long sgdg_mlp_num_params(const void* p) {
  if (!p) return 0;
  const Mlp& m = *(const Mlp*)p;
  long long n = 0;
  for (auto& L : m.l) n += (long long)L.fin * L.fout + L.fout;
  return n;
}

sgdg_status sgdg_mlp_get_params(const void* p, float* host) {
  if (!p || !host) return SGDG_EINVAL;
  const Mlp& m = *(const Mlp*)p;
  size_t o = 0;
  for (auto& L : m.l) {
    const size_t nw = (size_t)L.fin * L.fout;
    if (cudaMemcpy(host + o, L.W, 4 * nw, cudaMemcpyDeviceToHost) != cudaSuccess) return SGDG_ECUDA;
    o += nw;
    if (cudaMemcpy(host + o, L.b, 4 * L.fout, cudaMemcpyDeviceToHost) != cudaSuccess) return SGDG_ECUDA;
    o += L.fout;
  }
  return SGDG_OK;
}

sgdg_status sgdg_mlp_set_params(void* p, const float* host) {
  if (!p || !host) return SGDG_EINVAL;
  Mlp& m = *(Mlp*)p;
  size_t o = 0;
  for (auto& L : m.l) {
    const size_t nw = (size_t)L.fin * L.fout;
    if (cudaMemcpy(L.W, host + o, 4 * nw, cudaMemcpyHostToDevice) != cudaSuccess) return SGDG_ECUDA;
    o += nw;
    if (cudaMemcpy(L.b, host + o, 4 * L.fout, cudaMemcpyHostToDevice) != cudaSuccess) return SGDG_ECUDA;
    o += L.fout;
  }
  refresh_bf16(m, nullptr);
  return cudaDeviceSynchronize() == cudaSuccess ? SGDG_OK : SGDG_ECUDA;
}

}  // extern "C"
