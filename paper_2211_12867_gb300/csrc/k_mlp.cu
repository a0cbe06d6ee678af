// Learned refinement pre-flagger: features, forward, backward and Adam.
//
// The paper refines with criteria evaluated on the solution (Sect. 3); this
// predictor anticipates the estimator's next decision.  Per block: the
// index-space gradient magnitude of density, radial speed and pressure, each
// divided by the cell's magnitude, averaged over the three variables and over
// 4 x 4 x 4 sub-cubes -> 64 inputs; MLP 64 -> 128 (ReLU) -> 128 (ReLU) -> 1
// (sigmoid); binary cross-entropy; Adam.  FP32 storage and accumulation.  The
// layers are tiny (batch x 128 x 128), so they are plain FMA loops: one thread
// per hidden unit in the forward and backward vectors, one thread per
// parameter for the weight gradients (a fixed-order sum over the batch, so the
// gradient is deterministic).
#include "mhd_device.cuh"

#define MLP_IN 64
#define MLP_H 128

namespace {

struct MlpView {
  const float *W1, *b1, *W2, *b2, *w3, *b3;
};

__host__ __device__ inline MlpView mlp_view(const float *th) {
  MlpView m;
  m.W1 = th;
  m.b1 = m.W1 + MLP_H * MLP_IN;
  m.W2 = m.b1 + MLP_H;
  m.b2 = m.W2 + MLP_H * MLP_H;
  m.w3 = m.b2 + MLP_H;
  m.b3 = m.w3 + MLP_H;
  return m;
}

// One warp per sub-cube (4 x 4 x 4 sub-cubes of s0 x s1 x s2 cells with
// s = n / 4; cells past 4 s in a direction belong to none): the lanes take
// the sub-cube's cells in a fixed stride, add in FP64 and reduce in a fixed
// shuffle tree, so the features are the same bits on every run and for
// every member.
template <typename real>
__global__ void k_features(const KParams kp, const real *U, int slot0, float *out) {
  const int slot = slot0 + blockIdx.x;
  const int n0 = kp.nb[0], n1 = kp.nb[1], n2 = kp.nb[2];
  const int s0 = n0 / 4, s1 = n1 / 4, s2 = n2 / 4, per = s0 * s1 * s2;
  const double gm1 = kp.gamma - 1.0;
  auto cell = [&](int v, int i, int j, int k) -> double {
    return (double)U[((((size_t)slot * kp.nvs + v) * kp.P[0] + i) * kp.P[1] + j) * kp.P[2] + k];
  };
  auto prims = [&](int i, int j, int k, double *w) {  // rho, v_r, p
    const double r = cell(0, i, j, k), m1 = cell(1, i, j, k), m2 = cell(2, i, j, k), m3 = cell(3, i, j, k);
    const double b1 = cell(5, i, j, k), b2 = cell(6, i, j, k), b3 = cell(7, i, j, k);
    w[0] = r;
    w[1] = m1 / r;
    w[2] = gm1 * (cell(4, i, j, k) - 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) / r - 0.5 * (b1 * b1 + b2 * b2 + b3 * b3));
  };
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int sc = threadIdx.x >> 5; sc < 64; sc += nw) {
    const int a = sc / 16, b = (sc / 4) % 4, cc = sc % 4;
    double acc = 0.0;
    for (int t = lane; t < per; t += 32) {
      const int i = a * s0 + t / (s1 * s2), j = b * s1 + (t / s2) % s1, k = cc * s2 + t % s2;
      const int p0 = i + NGH, p1 = j + NGH, p2 = k + NGH;
      double w0[3], wm[3][3], wp[3][3];
      prims(p0, p1, p2, w0);
      prims(p0 - 1, p1, p2, wm[0]);
      prims(p0 + 1, p1, p2, wp[0]);
      prims(p0, p1 - 1, p2, wm[1]);
      prims(p0, p1 + 1, p2, wp[1]);
      prims(p0, p1, p2 - 1, wm[2]);
      prims(p0, p1, p2 + 1, wp[2]);
      double g = 0.0;
      for (int q = 0; q < 3; q++) {
        double s = 0.0;
        for (int d = 0; d < 3; d++) {
          const double cd = 0.5 * (wp[d][q] - wm[d][q]);
          s += cd * cd;
        }
        g += sqrt(s) / (fabs(w0[q]) + 1e-30);
      }
      acc += g / 3.0;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[(size_t)blockIdx.x * 64 + sc] = (float)(acc / per);
  }
}

// forward over rows of X (row index list `idx` or identity), 4 samples per CTA
constexpr int SPC = 4;
__global__ void k_forward(const float *theta, const float *X, const int *idx, int B, float *h1g, float *h2g,
                          float *y) {
  __shared__ float xs[SPC][MLP_IN];
  __shared__ float hs[SPC][MLP_H];
  __shared__ float red[SPC][MLP_H / 32];
  const MlpView m = mlp_view(theta);
  const int s0 = blockIdx.x * SPC, j = threadIdx.x;
  for (int e = j; e < SPC * MLP_IN; e += MLP_H) {
    const int s = e / MLP_IN, i = e % MLP_IN;
    const int row = s0 + s < B ? (idx ? idx[s0 + s] : s0 + s) : -1;
    xs[s][i] = row >= 0 ? X[(size_t)row * MLP_IN + i] : 0.f;
  }
  __syncthreads();
  float a[SPC];
  for (int s = 0; s < SPC; s++) a[s] = m.b1[j];
  for (int i = 0; i < MLP_IN; i++) {
    const float wv = m.W1[j * MLP_IN + i];
    for (int s = 0; s < SPC; s++) a[s] = fmaf(wv, xs[s][i], a[s]);
  }
  for (int s = 0; s < SPC; s++) {
    const float h = fmaxf(a[s], 0.f);
    hs[s][j] = h;
    if (s0 + s < B) h1g[(size_t)(s0 + s) * MLP_H + j] = h;
  }
  __syncthreads();
  for (int s = 0; s < SPC; s++) a[s] = m.b2[j];
  for (int k = 0; k < MLP_H; k++) {
    const float wv = m.W2[j * MLP_H + k];
    for (int s = 0; s < SPC; s++) a[s] = fmaf(wv, hs[s][k], a[s]);
  }
  float z[SPC];
  for (int s = 0; s < SPC; s++) {
    const float h = fmaxf(a[s], 0.f);
    if (s0 + s < B) h2g[(size_t)(s0 + s) * MLP_H + j] = h;
    z[s] = m.w3[j] * h;
  }
  for (int s = 0; s < SPC; s++) {
    float v = z[s];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((j & 31) == 0) red[s][j / 32] = v;
  }
  __syncthreads();
  if (j < SPC && s0 + j < B) {
    float zz = m.b3[0];
    for (int w = 0; w < MLP_H / 32; w++) zz += red[j][w];
    y[s0 + j] = 1.f / (1.f + expf(-zz));
  }
}

// per-sample backward vectors; loss accumulates the summed cross-entropy
__global__ void k_backvec(const float *theta, const float *T, const int *idx, int B, const float *h1g,
                          const float *h2g, const float *y, float *dz, float *dh2g, float *dh1g, float *loss) {
  __shared__ float d2[SPC][MLP_H];
  const MlpView m = mlp_view(theta);
  const int s0 = blockIdx.x * SPC, k = threadIdx.x;
  for (int s = 0; s < SPC; s++) {
    const int b = s0 + s;
    float dzz = 0.f;
    if (b < B) {
      const float t = T[idx ? idx[b] : b];
      dzz = (y[b] - t) / (float)B;
      if (k == 0) {
        dz[b] = dzz;
        const float yc = fminf(fmaxf(y[b], 1e-7f), 1.f - 1e-7f);
        atomicAdd(loss, -(t * logf(yc) + (1.f - t) * logf(1.f - yc)));
      }
      const float v = h2g[(size_t)b * MLP_H + k] > 0.f ? dzz * m.w3[k] : 0.f;
      d2[s][k] = v;
      dh2g[(size_t)b * MLP_H + k] = v;
    } else {
      d2[s][k] = 0.f;
    }
  }
  __syncthreads();
  float acc[SPC];
  for (int s = 0; s < SPC; s++) acc[s] = 0.f;
  for (int j = 0; j < MLP_H; j++) {
    const float wv = m.W2[j * MLP_H + k];
    for (int s = 0; s < SPC; s++) acc[s] = fmaf(wv, d2[s][j], acc[s]);
  }
  for (int s = 0; s < SPC; s++) {
    const int b = s0 + s;
    if (b < B) dh1g[(size_t)b * MLP_H + k] = h1g[(size_t)b * MLP_H + k] > 0.f ? acc[s] : 0.f;
  }
}

// parameter gradients: one thread per parameter, fixed-order sum over the batch
__global__ void k_wgrad(const float *X, const int *idx, int B, const float *h1g, const float *h2g,
                        const float *dz, const float *dh2g, const float *dh1g, float *grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int n1 = MLP_H * MLP_IN, n2 = n1 + MLP_H, n3 = n2 + MLP_H * MLP_H, n4 = n3 + MLP_H, n5 = n4 + MLP_H;
  if (p > n5) return;
  float s = 0.f;
  if (p < n1) {
    const int j = p / MLP_IN, i = p % MLP_IN;
    for (int b = 0; b < B; b++) s = fmaf(dh1g[(size_t)b * MLP_H + j], X[(size_t)(idx ? idx[b] : b) * MLP_IN + i], s);
  } else if (p < n2) {
    const int j = p - n1;
    for (int b = 0; b < B; b++) s += dh1g[(size_t)b * MLP_H + j];
  } else if (p < n3) {
    const int q = p - n2, j = q / MLP_H, k = q % MLP_H;
    for (int b = 0; b < B; b++) s = fmaf(dh2g[(size_t)b * MLP_H + j], h1g[(size_t)b * MLP_H + k], s);
  } else if (p < n4) {
    const int j = p - n3;
    for (int b = 0; b < B; b++) s += dh2g[(size_t)b * MLP_H + j];
  } else if (p < n5) {
    const int j = p - n4;
    for (int b = 0; b < B; b++) s = fmaf(dz[b], h2g[(size_t)b * MLP_H + j], s);
  } else {
    for (int b = 0; b < B; b++) s += dz[b];
  }
  grad[p] = s;
}

__global__ void k_adam(float *theta, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                       float eps, float bc1, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float gg = g[p];
  const float mm = b1 * m[p] + (1.f - b1) * gg;
  const float vv = b2 * v[p] + (1.f - b2) * gg * gg;
  m[p] = mm;
  v[p] = vv;
  theta[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
}

// combine: refine where the predictor says so, otherwise keep the plain flag
// learned pre-flag: probability above 1/2 on a block that can still refine
__global__ void k_combine(const float *prob, const DevBlock *blk, signed char *flags, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && prob[i] > 0.5f && blk[i].level < blk[i].lmax) flags[i] = 1;
}

}  // namespace

int mlp_n_params() { return MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1; }

void mlp_features_launch(const KParams &kp, const void *U, int precision, int slot0, int nslots, float *out,
                         cudaStream_t s) {
  if (nslots <= 0) return;
  if (precision)
    k_features<float><<<nslots, 256, 0, s>>>(kp, (const float *)U, slot0, out);
  else
    k_features<double><<<nslots, 256, 0, s>>>(kp, (const double *)U, slot0, out);
}

void mlp_forward_launch(const float *theta, const float *X, const int *idx, int B, float *h1, float *h2, float *y,
                        cudaStream_t s) {
  if (B <= 0) return;
  k_forward<<<(B + SPC - 1) / SPC, MLP_H, 0, s>>>(theta, X, idx, B, h1, h2, y);
}

void mlp_backward_launch(const float *theta, const float *X, const float *T, const int *idx, int B,
                         const float *h1, const float *h2, const float *y, float *dz, float *dh2, float *dh1,
                         float *grad, float *loss, cudaStream_t s) {
  if (B <= 0) return;
  k_backvec<<<(B + SPC - 1) / SPC, MLP_H, 0, s>>>(theta, T, idx, B, h1, h2, y, dz, dh2, dh1, loss);
  const int np = mlp_n_params();
  k_wgrad<<<(np + 255) / 256, 256, 0, s>>>(X, idx, B, h1, h2, dz, dh2, dh1, grad);
}

void mlp_adam_launch(float *theta, const float *g, float *m, float *v, float lr, int step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  const int np = mlp_n_params();
  k_adam<<<(np + 255) / 256, 256, 0, s>>>(theta, g, m, v, np, lr, b1, b2, 1e-8f, bc1, bc2);
}

void mlp_combine_launch(const float *prob, const DevBlock *blk, signed char *flags, int n, cudaStream_t s) {
  if (n > 0) k_combine<<<(n + 255) / 256, 256, 0, s>>>(prob, blk, flags, n);
}
