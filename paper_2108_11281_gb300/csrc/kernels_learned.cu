// Learned correction inside the multigrid cycle: a bias-free 3-layer 3x3
// convolutional network (channels c0 -> 16 -> 16 -> c0, ReLU after the first
// two layers) on the fine lattice, with its training kernels (backward data
// and weight gradients, the loss seed of ||A net(r) - r||^2 / ||r||^2, Adam).
// The paper has no learned component; this is the project's smoother.
//
// Activations are FP32 blocks [site][channel][k] (the k columns innermost, as
// for vectors).  Channel 2a / 2a+1 hold Re / Im of dof a for complex vectors,
// channel a holds dof a for real ones.  Weights are FP32 [c_out][c_in][3][3];
// tap (ty, tx) reads the site (i + tx - 1, j + ty - 1), periodic or zero
// outside a Dirichlet lattice.
#include "mlmc_internal.cuh"

namespace mlmc {

__device__ inline int tap_site(int i, int j, int tx, int ty, int nx, int ny, int periodic) {
  int ii = i + tx - 1, jj = j + ty - 1;
  if (periodic) {
    ii = ii < 0 ? ii + nx : (ii >= nx ? ii - nx : ii);
    jj = jj < 0 ? jj + ny : (jj >= ny ? jj - ny : jj);
    return jj * nx + ii;
  }
  if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) return -1;
  return jj * nx + ii;
}

// ------------------------------------------------------------------ vector <-> channels
template <class T>
__global__ void k_to_channels(const T *x, float *a, int nsite, int d, int k) {
  const int cpd = sizeof(T) == sizeof(double) * 2 || sizeof(T) == sizeof(float) * 2 ? 2 : 1;
  unsigned total = (unsigned)nsite * d * k;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    unsigned row = t / (unsigned)k;
    int c = (int)(t - row * (unsigned)k);
    int s = (int)(row / (unsigned)d), dof = (int)(row - (unsigned)s * d);
    T v = x[t];
    float* base = a + ((size_t)s * d * cpd) * k + c;
    if (cpd == 2) {
      base[(size_t)(2 * dof) * k] = (float)re(v);
      base[(size_t)(2 * dof + 1) * k] = (float)im(v);
    } else {
      base[(size_t)dof * k] = (float)re(v);
    }
  }
}

// x += from_channels(a)
template <class T>
__global__ void k_add_from_channels(T *x, const float *a, int nsite, int d, int k) {
  const int cpd = sizeof(T) == sizeof(double) * 2 || sizeof(T) == sizeof(float) * 2 ? 2 : 1;
  unsigned total = (unsigned)nsite * d * k;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    unsigned row = t / (unsigned)k;
    int c = (int)(t - row * (unsigned)k);
    int s = (int)(row / (unsigned)d), dof = (int)(row - (unsigned)s * d);
    const float *base = a + ((size_t)s * d * cpd) * k + c;
    if (cpd == 2) x[t] = x[t] + make<T>(base[(size_t)(2 * dof) * k], base[(size_t)(2 * dof + 1) * k]);
    else x[t] = x[t] + make<T>(base[(size_t)dof * k], 0.0);
  }
}

// ------------------------------------------------------------------ convolution forward
// out[s][co][c] = act(sum_{tap, ci} W[co][ci][tap] in[tap_site(s)][ci][c]); one thread per (site, column).
template <int CI, int CO, bool RELU>
__global__ void __launch_bounds__(256) k_conv_fwd(const float *__restrict__ in, const float *__restrict__ W,
                                                  float *__restrict__ out, int nx, int ny, int k, int periodic) {
  // weights transposed to [tap][ci][co] so that 4 outputs take one 16-byte shared load
  __shared__ __align__(16) float Ws[9 * CI * CO];
  for (int i = threadIdx.x; i < CO * CI * 9; i += blockDim.x) {
    int co = i / (CI * 9), ci = (i / 9) % CI, tap = i % 9;
    Ws[(tap * CI + ci) * CO + co] = W[i];
  }
  __syncthreads();
  const unsigned total = (unsigned)nx * ny * k;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int s = (int)(t / (unsigned)k);
    const int c = (int)(t - (unsigned)s * k);
    const int i = s % nx, j = s / nx;
    float acc[CO];
#pragma unroll
    for (int co = 0; co < CO; ++co) acc[co] = 0.f;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      int nb = tap_site(i, j, tap % 3, tap / 3, nx, ny, periodic);
      if (nb < 0) continue;
      const float *src = in + (size_t)nb * CI * k + c;
#pragma unroll
      for (int ci = 0; ci < CI; ++ci) {
        float v = src[(size_t)ci * k];
        const float *w = Ws + (tap * CI + ci) * CO;
        if constexpr (CO % 4 == 0) {
#pragma unroll
          for (int co = 0; co < CO; co += 4) {
            float4 w4 = *reinterpret_cast<const float4 *>(w + co);
            acc[co] = fmaf(w4.x, v, acc[co]);
            acc[co + 1] = fmaf(w4.y, v, acc[co + 1]);
            acc[co + 2] = fmaf(w4.z, v, acc[co + 2]);
            acc[co + 3] = fmaf(w4.w, v, acc[co + 3]);
          }
        } else {
#pragma unroll
          for (int co = 0; co < CO; ++co) acc[co] = fmaf(w[co], v, acc[co]);
        }
      }
    }
    float *dst = out + (size_t)s * CO * k + c;
#pragma unroll
    for (int co = 0; co < CO; ++co) dst[(size_t)co * k] = RELU ? fmaxf(acc[co], 0.f) : acc[co];
  }
}

// ------------------------------------------------------------------ backward: data
// gin[s][ci][c] = mask(s, ci, c) * sum_{tap, co} W[co][ci][tap] gout[s'][co][c], where s' is the
// site whose tap `tap` reads s (s' = s shifted by the opposite offset).  mask = (act[s][ci][c] > 0)
// when `act` is given (ReLU of the layer that produced the input), else 1.
template <int CI, int CO>
__global__ void __launch_bounds__(256) k_conv_bwd_data(const float *__restrict__ gout, const float *__restrict__ W,
                                                       const float *__restrict__ act, float *__restrict__ gin, int nx,
                                                       int ny, int k, int periodic) {
  // weights transposed to [tap][co][ci]: 4 inputs take one 16-byte shared load
  __shared__ __align__(16) float Ws[9 * CO * CI];
  for (int i = threadIdx.x; i < CO * CI * 9; i += blockDim.x) {
    int co = i / (CI * 9), ci = (i / 9) % CI, tap = i % 9;
    Ws[(tap * CO + co) * CI + ci] = W[i];
  }
  __syncthreads();
  const unsigned total = (unsigned)nx * ny * k;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int s = (int)(t / (unsigned)k);
    const int c = (int)(t - (unsigned)s * k);
    const int i = s % nx, j = s / nx;
    float acc[CI];
#pragma unroll
    for (int ci = 0; ci < CI; ++ci) acc[ci] = 0.f;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      // s' with tap_site(s', tap) = s: offset (1 - tx, 1 - ty) from s
      int nb = tap_site(i, j, 2 - tap % 3, 2 - tap / 3, nx, ny, periodic);
      if (nb < 0) continue;
      const float *src = gout + (size_t)nb * CO * k + c;
#pragma unroll
      for (int co = 0; co < CO; ++co) {
        float g = src[(size_t)co * k];
        const float *w = Ws + (tap * CO + co) * CI;
        if constexpr (CI % 4 == 0) {
#pragma unroll
          for (int ci = 0; ci < CI; ci += 4) {
            float4 w4 = *reinterpret_cast<const float4 *>(w + ci);
            acc[ci] = fmaf(w4.x, g, acc[ci]);
            acc[ci + 1] = fmaf(w4.y, g, acc[ci + 1]);
            acc[ci + 2] = fmaf(w4.z, g, acc[ci + 2]);
            acc[ci + 3] = fmaf(w4.w, g, acc[ci + 3]);
          }
        } else {
#pragma unroll
          for (int ci = 0; ci < CI; ++ci) acc[ci] = fmaf(w[ci], g, acc[ci]);
        }
      }
    }
    float *dst = gin + (size_t)s * CI * k + c;
#pragma unroll
    for (int ci = 0; ci < CI; ++ci) {
      float m = act ? (act[(size_t)s * CI * k + (size_t)ci * k + c] > 0.f ? 1.f : 0.f) : 1.f;
      dst[(size_t)ci * k] = acc[ci] * m;
    }
  }
}

// ------------------------------------------------------------------ backward: weights
// partial[block][co][ci][tap] = sum over the block's (site, column) pairs of
// gout[s][co][c] * in[tap_site(s)][ci][c].  Pairs are staged through shared
// memory in tiles; each thread owns a fixed set of weight entries, so the
// per-block sums are deterministic.  Then k_weight_reduce adds the blocks in order.
template <int CI, int CO>
__global__ void __launch_bounds__(256) k_conv_bwd_weight(const float *__restrict__ in, const float *__restrict__ gout,
                                                         float *__restrict__ partial, int nx, int ny, int k,
                                                         int periodic) {
  constexpr int NW = CO * CI * 9;
  constexpr int TP = 32;                       // pairs per tile
  constexpr int PER = (NW + 255) / 256;        // weight entries per thread
  __shared__ float g_t[TP][CO];
  __shared__ float x_t[TP][9][CI];
  float acc[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) acc[q] = 0.f;
  const unsigned total = (unsigned)nx * ny * k;
  const unsigned per_block = (total + gridDim.x - 1) / gridDim.x;
  const unsigned p0 = blockIdx.x * per_block;
  const unsigned p1 = p0 + per_block < total ? p0 + per_block : total;
  for (unsigned base = p0; base < p1; base += TP) {
    // stage TP pairs
    for (int e = threadIdx.x; e < TP * (CO + 9 * CI); e += blockDim.x) {
      int p = e / (CO + 9 * CI), r = e % (CO + 9 * CI);
      unsigned t = base + p;
      float v = 0.f;
      if (t < p1) {
        int s = (int)(t / (unsigned)k), c = (int)(t - (unsigned)s * k);
        if (r < CO) {
          v = gout[(size_t)s * CO * k + (size_t)r * k + c];
        } else {
          int q = r - CO, tap = q / CI, ci = q % CI;
          int nb = tap_site(s % nx, s / nx, tap % 3, tap / 3, nx, ny, periodic);
          v = nb < 0 ? 0.f : in[(size_t)nb * CI * k + (size_t)ci * k + c];
        }
      }
      if (r < CO) g_t[p][r] = v;
      else x_t[p][(r - CO) / CI][(r - CO) % CI] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      int w = threadIdx.x + q * 256;
      if (w < NW) {
        int co = w / (CI * 9), ci = (w / 9) % CI, tap = w % 9;
        float a = acc[q];
        for (int p = 0; p < TP; ++p) a = fmaf(g_t[p][co], x_t[p][tap][ci], a);
        acc[q] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    int w = threadIdx.x + q * 256;
    if (w < NW) partial[(size_t)blockIdx.x * NW + w] = acc[q];
  }
}

__global__ void k_weight_reduce(const float *partial, int nblocks, int nw, float *grad, float scale) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nw) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += (double)partial[(size_t)b * nw + w];
  grad[w] = (float)(s * scale);
}

// ------------------------------------------------------------------ Adam
__global__ void k_adam(float *W, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float mi = b1 * m[i] + (1.f - b1) * g[i];
  float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  W[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------------------ launchers
static unsigned cgrid(unsigned total) {
  unsigned g = (total + 255) / 256;
  return g < 152 * 16 ? (g ? g : 1) : 152 * 16;
}

void launch_to_channels(DType t, const void *x, float *a, int nsite, int d, int k, cudaStream_t s) {
  unsigned g = cgrid((unsigned)nsite * d * k);
  MLMC_DISPATCH(t, T, k_to_channels<T><<<g, 256, 0, s>>>((const T *)x, a, nsite, d, k));
  MLMC_LAUNCH_CHECK("k_to_channels");
}

void launch_add_from_channels(DType t, void *x, const float *a, int nsite, int d, int k, cudaStream_t s) {
  unsigned g = cgrid((unsigned)nsite * d * k);
  MLMC_DISPATCH(t, T, k_add_from_channels<T><<<g, 256, 0, s>>>((T *)x, a, nsite, d, k));
  MLMC_LAUNCH_CHECK("k_add_from_channels");
}

#define MLMC_CONV_SHAPES(X) X(1, 16) X(2, 16) X(4, 16) X(16, 16) X(16, 1) X(16, 2) X(16, 4)

void launch_conv_fwd(int ci, int co, bool relu, const float *in, const float *W, float *out, int nx, int ny, int k,
                     int periodic, cudaStream_t s) {
  unsigned g = cgrid((unsigned)nx * ny * k);
#define MLMC_FWD(A, B)                                                                                        \
  if (ci == A && co == B) {                                                                                   \
    if (relu) k_conv_fwd<A, B, true><<<g, 256, 0, s>>>(in, W, out, nx, ny, k, periodic);                      \
    else k_conv_fwd<A, B, false><<<g, 256, 0, s>>>(in, W, out, nx, ny, k, periodic);                          \
    MLMC_LAUNCH_CHECK("k_conv_fwd");                                                                          \
    return;                                                                                                   \
  }
  MLMC_CONV_SHAPES(MLMC_FWD)
#undef MLMC_FWD
  throw cuda_error{cudaErrorInvalidValue, "conv: unsupported channel counts"};
}

void launch_conv_bwd_data(int ci, int co, const float *gout, const float *W, const float *act, float *gin, int nx,
                          int ny, int k, int periodic, cudaStream_t s) {
  unsigned g = cgrid((unsigned)nx * ny * k);
#define MLMC_BWD(A, B)                                                                                        \
  if (ci == A && co == B) {                                                                                   \
    k_conv_bwd_data<A, B><<<g, 256, 0, s>>>(gout, W, act, gin, nx, ny, k, periodic);                          \
    MLMC_LAUNCH_CHECK("k_conv_bwd_data");                                                                     \
    return;                                                                                                   \
  }
  MLMC_CONV_SHAPES(MLMC_BWD)
#undef MLMC_BWD
  throw cuda_error{cudaErrorInvalidValue, "conv: unsupported channel counts"};
}

int conv_weight_blocks() { return 152 * 2; }

void launch_conv_bwd_weight(int ci, int co, const float *in, const float *gout, float *partial, float *grad,
                            float scale, int nx, int ny, int k, int periodic, cudaStream_t s) {
  int nb = conv_weight_blocks();
  int nw = ci * co * 9;
#define MLMC_BWW(A, B)                                                                                        \
  if (ci == A && co == B) {                                                                                   \
    k_conv_bwd_weight<A, B><<<nb, 256, 0, s>>>(in, gout, partial, nx, ny, k, periodic);                       \
    MLMC_LAUNCH_CHECK("k_conv_bwd_weight");                                                                   \
    k_weight_reduce<<<(nw + 127) / 128, 128, 0, s>>>(partial, nb, nw, grad, scale);                           \
    MLMC_LAUNCH_CHECK("k_weight_reduce");                                                                     \
    return;                                                                                                   \
  }
  MLMC_CONV_SHAPES(MLMC_BWW)
#undef MLMC_BWW
  throw cuda_error{cudaErrorInvalidValue, "conv: unsupported channel counts"};
}

void launch_weight_reduce(const float *partial, int nblocks, int nw, float *grad, float scale, cudaStream_t s) {
  k_weight_reduce<<<(nw + 127) / 128, 128, 0, s>>>(partial, nblocks, nw, grad, scale);
  MLMC_LAUNCH_CHECK("k_weight_reduce");
}

void launch_adam(float *W, const float *g, float *m, float *v, int n, float lr, int step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<(n + 255) / 256, 256, 0, s>>>(W, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
  MLMC_LAUNCH_CHECK("k_adam");
}

// J v: negate the second half of each site's dofs (spin parity of Example 5.3)
template <class T>
__global__ void k_spin_flip(T *x, int nsite, int d, int k) {
  unsigned total = (unsigned)nsite * d * k;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    unsigned row = t / (unsigned)k;
    int dof = (int)(row % (unsigned)d);
    if (dof >= d / 2) x[t] = -x[t];
  }
}

void launch_spin_flip(DType t, void *x, int nsite, int d, int k, cudaStream_t s) {
  unsigned g = cgrid((unsigned)nsite * d * k);
  MLMC_DISPATCH(t, T, k_spin_flip<T><<<g, 256, 0, s>>>((T *)x, nsite, d, k));
  MLMC_LAUNCH_CHECK("k_spin_flip");
}

}  // namespace mlmc
