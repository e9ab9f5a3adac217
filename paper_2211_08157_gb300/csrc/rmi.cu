// Learned index over the sorted kept keys (a recursive model index, RMI).
//
// Root: a 1 -> 32 -> 1 ReLU MLP maps the normalised key x = (key - kmin) /
// (kmax - kmin) to the normalised rank; leaf = floor(root(x) * n_leaves).
// It is trained on the GPU by the kernels below (forward + backward with a
// fixed-shape reduction, then an Adam step) on evenly spaced keys of the index.
// Leaves: per leaf a least-squares line rank ~ slope * (key - base) + icept
// over the keys the root routes there (sums in double, parameters stored in
// FP32), and an error bound eps = max |rank - prediction| over those keys,
// computed with the same FP32 device functions the lookup uses, so that the
// last-mile search in [pred - eps, pred + eps] always finds a present key.
// Leaves with eps above the threshold route their queries to the hash table.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "rmi_device.cuh"

namespace god {
namespace {

constexpr int H = kRootHidden;
constexpr int NP = 3 * H + 1;      // W1, b1, W2, b2
constexpr int kGradThreads = 256;
constexpr int kGradBlocks = 64;    // fixed: the reduction shape (and so the FP32 result) never changes

// Per-block partial gradients (and loss) of mean((f(x) - y)^2) over the
// samples i = block*256 + tid + k*(blocks*256). Deterministic: fixed warp
// shuffle trees, then warps summed in index order.
__global__ void __launch_bounds__(kGradThreads) root_grad_partial(const float* __restrict__ theta,
                                                                  const float* __restrict__ xs,
                                                                  const float* __restrict__ ys, uint64_t n,
                                                                  float inv_n, float* __restrict__ partial) {
  __shared__ float sp[NP];
  __shared__ float warp_part[kGradThreads / 32][NP + 1];
  for (int i = threadIdx.x; i < NP; i += kGradThreads) sp[i] = theta[i];
  __syncthreads();
  float g[NP + 1];
#pragma unroll
  for (int i = 0; i < NP + 1; ++i) g[i] = 0.0f;
  const uint64_t stride = (uint64_t)gridDim.x * kGradThreads;
  for (uint64_t i = (uint64_t)blockIdx.x * kGradThreads + threadIdx.x; i < n; i += stride) {
    const float x = xs[i];
    float a[H];
    float f = sp[3 * H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
      a[h] = fmaxf(__fmaf_rn(sp[h], x, sp[H + h]), 0.0f);
      f = __fmaf_rn(sp[2 * H + h], a[h], f);
    }
    const float e = __fsub_rn(f, ys[i]);
    g[NP] = __fadd_rn(g[NP], __fmul_rn(e, e));
    const float de = __fmul_rn(__fmul_rn(2.0f, e), inv_n);
#pragma unroll
    for (int h = 0; h < H; ++h) {
      g[2 * H + h] = __fadd_rn(g[2 * H + h], __fmul_rn(de, a[h]));
      if (a[h] > 0.0f) {
        const float dpre = __fmul_rn(de, sp[2 * H + h]);
        g[h] = __fadd_rn(g[h], __fmul_rn(dpre, x));
        g[H + h] = __fadd_rn(g[H + h], dpre);
      }
    }
    g[3 * H] = __fadd_rn(g[3 * H], de);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NP + 1; ++i) {
    float v = g[i];
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, d));
    if (lane == 0) warp_part[wid][i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NP + 1; i += kGradThreads) {
    float v = 0.0f;
    for (int w = 0; w < kGradThreads / 32; ++w) v = __fadd_rn(v, warp_part[w][i]);
    partial[(uint64_t)blockIdx.x * (NP + 1) + i] = v;
  }
}

// Sums the per-block partials in block order; optionally applies one Adam step.
__global__ void root_reduce_adam(const float* __restrict__ partial, int blocks, float* __restrict__ grad_out,
                                 float* __restrict__ theta, float* __restrict__ m1, float* __restrict__ m2, int step,
                                 float lr, int apply, float inv_n) {
  const int i = threadIdx.x;
  if (i > NP) return;
  float v = 0.0f;
  for (int b = 0; b < blocks; ++b) v = __fadd_rn(v, partial[(uint64_t)b * (NP + 1) + i]);
  if (i == NP) v = __fmul_rn(v, inv_n);  // loss = mean squared error
  if (grad_out) grad_out[i] = v;
  if (apply && i < NP) {
    const float b1 = 0.9f, b2 = 0.999f;
    m1[i] = b1 * m1[i] + (1.0f - b1) * v;
    m2[i] = b2 * m2[i] + (1.0f - b2) * v * v;
    const float mh = m1[i] / (1.0f - powf(b1, (float)step));
    const float vh = m2[i] / (1.0f - powf(b2, (float)step));
    theta[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
  }
}

// Least-squares readout: with the hidden layer fixed, the output layer (W2,
// b2) that minimises the MSE solves the normal equations G w = r with
// G = sum phi phi^T, r = sum phi y, phi = (relu(W1 x + b1), 1). Entries of the
// upper triangle of G, then r, are accumulated in double per sample chunk
// (fixed order: deterministic).
constexpr int kGramN = H + 1;
constexpr int kGramTri = kGramN * (kGramN + 1) / 2;
constexpr int kGramE = kGramTri + kGramN;
constexpr int kGramChunks = 256;

__device__ __forceinline__ double phi_of(const float* th, float x, int h) {
  if (h == H) return 1.0;
  return (double)fmaxf(__fmaf_rn(th[h], x, th[H + h]), 0.0f);
}

__global__ void root_gram_partial(const float* __restrict__ theta, const float* __restrict__ xs,
                                  const float* __restrict__ ys, uint64_t n, double* __restrict__ partial) {
  __shared__ float th[NP];
  for (int i = threadIdx.x; i < NP; i += blockDim.x) th[i] = theta[i];
  __syncthreads();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kGramE) return;
  int i = 0, j = 0;
  if (e < kGramTri) {  // row-major upper triangle
    int rem = e;
    while (rem >= kGramN - i) { rem -= kGramN - i; ++i; }
    j = i + rem;
  } else {
    i = e - kGramTri;
    j = -1;  // r entry
  }
  const uint64_t chunk = (n + kGramChunks - 1) / kGramChunks;
  const uint64_t lo = blockIdx.y * chunk, hi = min(n, lo + chunk);
  double acc = 0.0;
  for (uint64_t t = lo; t < hi; ++t) {
    const float x = xs[t];
    const double a = phi_of(th, x, i);
    acc += j >= 0 ? a * phi_of(th, x, j) : a * (double)ys[t];
  }
  partial[(uint64_t)blockIdx.y * kGramE + e] = acc;
}

// Sum the chunk partials in order (one thread per entry), then one thread
// adds a tiny ridge, factors G = L L^T (Cholesky, shared memory) and solves;
// (W2, b2) go into theta.
__global__ void root_gram_solve(const double* __restrict__ partial, float* __restrict__ theta) {
  __shared__ double G[kGramN][kGramN + 1];
  __shared__ double r[kGramN], y[kGramN];
  for (int e = threadIdx.x; e < kGramE; e += blockDim.x) {
    double v = 0.0;
    for (int c = 0; c < kGramChunks; ++c) v += partial[(uint64_t)c * kGramE + e];
    if (e < kGramTri) {
      int i = 0, rem = e;
      while (rem >= kGramN - i) { rem -= kGramN - i; ++i; }
      G[i][i + rem] = v;
      G[i + rem][i] = v;
    } else {
      r[e - kGramTri] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double tr = 0.0;
  for (int i = 0; i < kGramN; ++i) tr += G[i][i];
  const double ridge = 1e-12 * tr / kGramN + 1e-300;
  for (int i = 0; i < kGramN; ++i) G[i][i] += ridge;
  for (int j = 0; j < kGramN; ++j) {
    double d = G[j][j];
    for (int k2 = 0; k2 < j; ++k2) d -= G[j][k2] * G[j][k2];
    d = d > 0 ? sqrt(d) : 1e-150;
    G[j][j] = d;
    for (int i = j + 1; i < kGramN; ++i) {
      double v = G[i][j];
      for (int k2 = 0; k2 < j; ++k2) v -= G[i][k2] * G[j][k2];
      G[i][j] = v / d;
    }
  }
  for (int i = 0; i < kGramN; ++i) {
    double v = r[i];
    for (int k2 = 0; k2 < i; ++k2) v -= G[i][k2] * y[k2];
    y[i] = v / G[i][i];
  }
  for (int i = kGramN - 1; i >= 0; --i) {
    double v = y[i];
    for (int k2 = i + 1; k2 < kGramN; ++k2) v -= G[k2][i] * y[k2];
    y[i] = v / G[i][i];
  }
  for (int h = 0; h < H; ++h) theta[2 * H + h] = (float)y[h];
  theta[3 * H] = (float)y[H];
}

__global__ void copy_floats(const float* src, float* dst, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Training samples: evenly spaced ranks r_i = floor(i * U / S); x = normalised
// key with the lookup's own FP32 expression; y = r_i / U.
__global__ void make_samples(const uint64_t* keys, uint64_t U, uint64_t S, uint64_t kmin, float inv_span, float* xs,
                             float* ys) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < S; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = (uint64_t)(((unsigned __int128)i * U) / S);
    xs[i] = __fmul_rn(__ull2float_rn(keys[r] - kmin), inv_span);
    ys[i] = (float)((double)r / (double)U);
  }
}

__global__ void route_keys(const RmiRoot* __restrict__ root, const uint64_t* __restrict__ keys, uint64_t U,
                           uint64_t* leaf_key, uint64_t* rank_val) {
  __shared__ RmiRoot R;
  if (threadIdx.x == 0) R = *root;
  __syncthreads();
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < U; r += (uint64_t)gridDim.x * blockDim.x) {
    leaf_key[r] = rmi_root_leaf(R, keys[r]);
    rank_val[r] = r;
  }
}

// lo/hi: [first, last + 1) of each leaf's run in the leaf-sorted order.
__global__ void leaf_bounds(const uint64_t* leaf_sorted, uint64_t U, uint32_t* lo, uint32_t* hi) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < U; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t l = leaf_sorted[i];
    if (i == 0 || leaf_sorted[i - 1] != l) lo[l] = (uint32_t)i;
    if (i == U - 1 || leaf_sorted[i + 1] != l) hi[l] = (uint32_t)(i + 1);
  }
}

// One thread per leaf: least squares in double over the leaf's keys (ranks
// ascend inside the run, so the first key is the smallest = base), then the
// error bound with the FP32 prediction of the lookup path.
__global__ void fit_leaves(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ ranks,
                           const uint32_t* __restrict__ lo, const uint32_t* __restrict__ hi, uint32_t n_leaves,
                           RmiLeaf* leaves, unsigned long long* stats) {
  unsigned long long eps_sum = 0;
  for (uint64_t l = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; l < n_leaves; l += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t b = lo[l], e = hi[l];
    RmiLeaf out;
    if (e <= b) {
      out.base_eps = 0;
      out.slope = 0.0f;
      out.icept = 0.0f;
      leaves[l] = out;
      continue;
    }
    const uint64_t base = keys[ranks[b]];
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (uint32_t i = b; i < e; ++i) {
      const uint64_t r = ranks[i];
      const double dx = (double)(keys[r] - base);
      const double dy = (double)r;
      sx += dx; sy += dy; sxx += dx * dx; sxy += dx * dy;
    }
    const double c = (double)(e - b);
    double slope = 0.0, icept = sy / c;
    const double den = c * sxx - sx * sx;
    if (e - b > 1 && den > 0) {
      slope = (c * sxy - sx * sy) / den;
      icept = (sy - slope * sx) / c;
    }
    const float fs = (float)slope, fi = (float)icept;
    uint64_t mx = 0;
    for (uint32_t i = b; i < e; ++i) {
      const uint64_t r = ranks[i];
      const int64_t p = rmi_leaf_pred(fs, fi, base, keys[r]);
      const int64_t d = p > (int64_t)r ? p - (int64_t)r : (int64_t)r - p;
      mx = max(mx, (uint64_t)d);
    }
    const uint64_t eps = mx > 255 ? 255 : mx;
    out.base_eps = (base & ((1ULL << 56) - 1)) | (eps << 56);
    out.slope = fs;
    out.icept = fi;
    leaves[l] = out;
    eps_sum += (unsigned long long)mx * (e - b);   // key-weighted eps sum
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) eps_sum += __shfl_xor_sync(0xffffffffu, eps_sum, d);
  if ((threadIdx.x & 31) == 0 && eps_sum) atomicAdd(&stats[0], eps_sum);
}

__global__ void leaf_stats(const RmiLeaf* leaves, const uint32_t* lo, const uint32_t* hi, uint32_t n_leaves,
                           uint32_t eps_max, unsigned long long* stats) {
  unsigned long long fl = 0, fk = 0, mx = 0;
  for (uint64_t l = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; l < n_leaves; l += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t cnt = hi[l] > lo[l] ? hi[l] - lo[l] : 0;
    const uint32_t eps = (uint32_t)(leaves[l].base_eps >> 56);
    if (cnt > 0 && eps > eps_max) {
      fl += 1;      // fallback leaves
      fk += cnt;    // keys in fallback leaves
    } else if (cnt > 0) {
      mx = max(mx, (unsigned long long)eps);  // largest bound used
    }
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    fl += __shfl_xor_sync(0xffffffffu, fl, d);
    fk += __shfl_xor_sync(0xffffffffu, fk, d);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
  }
  if ((threadIdx.x & 31) == 0) {
    if (fl) atomicAdd(&stats[3], fl);
    if (fk) atomicAdd(&stats[4], fk);
    if (mx) atomicMax(&stats[5], mx);
  }
}

// flag = 1 when the routed leaf ids of the (ascending) keys ever decrease.
__global__ void leaf_monotone(const uint64_t* leaf, uint64_t U, int* flag) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i + 1 < U; i += (uint64_t)gridDim.x * blockDim.x)
    if (leaf[i] > leaf[i + 1]) *flag = 1;
}

}  // namespace

// The network f(x) = b2 + sum_h W2[h] relu(W1[h] x + b1[h]) is linear between
// consecutive hinge points -b1[h] / W1[h]; on each piece the active units are
// those with W1[h] x + b1[h] > 0 at an interior point, A = sum of W2 W1 and
// C = b2 + sum of W2 b1 over them (units with W1 = 0 add W2 relu(b1) to every
// piece). Built in double, stored in FP32.
void rmi_root_pieces(RmiRoot& R) {
  double hs[kRootHidden];
  int nh = 0;
  for (int h = 0; h < kRootHidden; ++h) {
    if (R.W1[h] == 0.0f) continue;
    const double t = -(double)R.b1[h] / (double)R.W1[h];
    if (std::isfinite(t)) hs[nh++] = t;
  }
  std::sort(hs, hs + nh);
  for (int i = 0; i < kRootHidden; ++i) R.hx[i] = i < nh ? (float)hs[i] : INFINITY;
  for (int i = 0; i <= kRootHidden; ++i) {
    if (i > nh) {
      R.A[i] = R.A[nh];
      R.C[i] = R.C[nh];
      continue;
    }
    double mid;
    if (nh == 0) mid = 0.0;
    else if (i == 0) mid = hs[0] - 1.0;
    else if (i == nh) mid = hs[nh - 1] + 1.0;
    else mid = 0.5 * (hs[i - 1] + hs[i]);
    double A = 0.0, C = R.b2;
    for (int h = 0; h < kRootHidden; ++h) {
      if (R.W1[h] == 0.0f) {
        C += (double)R.W2[h] * std::max(0.0, (double)R.b1[h]);
      } else if ((double)R.W1[h] * mid + (double)R.b1[h] > 0.0) {
        A += (double)R.W2[h] * R.W1[h];
        C += (double)R.W2[h] * R.b1[h];
      }
    }
    R.A[i] = (float)A;
    R.C[i] = (float)C;
  }
}

namespace {

void init_root(RmiRoot* R, int kind) {
  // Knots of a piecewise-linear basis on [0, 1]: hidden unit h = relu(x - h/H);
  // output weights drawn from a fixed-seed generator (splitmix64). The linear
  // root (no network) keeps only f(x) = relu(x) = x.
  uint64_t s = 0x9E3779B97F4A7C15ULL;
  auto next = [&]() {
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int h = 0; h < H; ++h) {
    R->W1[h] = 1.0f;
    R->b1[h] = -(float)h / (float)H;
    R->W2[h] = (float)((next() - 0.5) * 0.5);
  }
  R->b2 = 0.0f;
  if (kind == GOD_ROOT_LINEAR) {
    for (int h = 0; h < H; ++h) { R->W1[h] = 0.0f; R->b1[h] = 0.0f; R->W2[h] = 0.0f; }
    R->W1[0] = 1.0f;
    R->W2[0] = 1.0f;
  }
}

}  // namespace

int rmi_root_grad_device(const float* d_theta, int Hh, const float* d_x, const float* d_y, uint64_t n, float* d_grad,
                         float* d_loss, cudaStream_t st) {
  if (Hh != H) {
    set_error("root hidden width must be 32");
    return GOD_EINVAL;
  }
  DBuf<float> partial, out;
  GOD_TRY(partial.alloc((size_t)kGradBlocks * (NP + 1), st));
  GOD_TRY(out.alloc(NP + 1, st));
  const float inv_n = n ? 1.0f / (float)n : 0.0f;
  GOD_LAUNCH(root_grad_partial, kGradBlocks, kGradThreads, 0, st, d_theta, d_x, d_y, n, inv_n, partial.p);
  GOD_LAUNCH(root_reduce_adam, 1, 128, 0, st, partial.p, kGradBlocks, out.p, nullptr, nullptr, nullptr, 0, 0.0f, 0,
             inv_n);
  GOD_CK(cudaMemcpyAsync(d_grad, out.p, NP * sizeof(float), cudaMemcpyDeviceToDevice, st));
  GOD_CK(cudaMemcpyAsync(d_loss, out.p + NP, sizeof(float), cudaMemcpyDeviceToDevice, st));
  return GOD_OK;
}

int build_rmi(god_index* idx, cudaStream_t st) {
  const uint64_t U = idx->n_keys;
  idx->has_rmi = 0;
  if (U == 0) return GOD_OK;
  const god_params& P = idx->params;
  int bits = P.rmi_leaf_bits;
  if (bits <= 0) {
    bits = 16;
    while (bits < 20 && (U >> bits) > 8) ++bits;
  }
  bits = std::max(16, std::min(20, bits));
  const uint32_t n_leaves = 1u << bits;
  RmiRoot R{};
  uint64_t kk[2];
  GOD_CK(cudaMemcpyAsync(&kk[0], idx->d_keys, 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaMemcpyAsync(&kk[1], idx->d_keys + U - 1, 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  R.kmin = kk[0];
  R.kmax = kk[1];
  R.inv_span = (R.kmax > R.kmin) ? (float)(1.0 / (double)(R.kmax - R.kmin)) : 0.0f;
  R.n_leaves = n_leaves;
  init_root(&R, P.rmi_root);

  DBuf<RmiRoot> d_root;
  GOD_TRY(d_root.alloc(1, st));
  float loss = 0.0f;
  if (P.rmi_root == GOD_ROOT_MLP) {   // the least-squares readout always; then rmi_train_steps Adam steps
    const uint64_t S = std::min<uint64_t>(U, std::max<uint32_t>(P.rmi_train_samples, 1));
    DBuf<float> xs, ys, theta, m1, m2, partial, gout;
    GOD_TRY(xs.alloc(S, st));
    GOD_TRY(ys.alloc(S, st));
    GOD_TRY(theta.alloc(NP, st));
    GOD_TRY(m1.alloc(NP, st));
    GOD_TRY(m2.alloc(NP, st));
    GOD_TRY(partial.alloc((size_t)kGradBlocks * (NP + 1), st));
    GOD_TRY(gout.alloc(NP + 1, st));
    GOD_LAUNCH(make_samples, (unsigned)std::min<uint64_t>((S + 255) / 256, 4096), 256, 0, st, idx->d_keys, U, S,
               R.kmin, R.inv_span, xs.p, ys.p);
    float th[NP];
    for (int h = 0; h < H; ++h) { th[h] = R.W1[h]; th[H + h] = R.b1[h]; th[2 * H + h] = R.W2[h]; }
    th[3 * H] = R.b2;
    GOD_CK(cudaMemcpyAsync(theta.p, th, sizeof(th), cudaMemcpyHostToDevice, st));
    GOD_CK(cudaMemsetAsync(m1.p, 0, NP * sizeof(float), st));
    GOD_CK(cudaMemsetAsync(m2.p, 0, NP * sizeof(float), st));
    const float inv_n = 1.0f / (float)S;
    const int steps = P.rmi_train_steps > 0 ? P.rmi_train_steps : 0;
    // 1. exact least-squares output layer over the fixed ReLU features
    DBuf<double> gpart;
    DBuf<float> best, gbest;
    GOD_TRY(gpart.alloc((size_t)kGramChunks * kGramE, st));
    GOD_TRY(best.alloc(NP, st));
    GOD_TRY(gbest.alloc(NP + 1, st));
    GOD_LAUNCH(root_gram_partial, dim3((kGramE + 255) / 256, kGramChunks), 256, 0, st, theta.p, xs.p, ys.p, S,
               gpart.p);
    GOD_LAUNCH(root_gram_solve, 1, 256, 0, st, gpart.p, theta.p);
    GOD_LAUNCH(copy_floats, 1, 128, 0, st, theta.p, best.p, NP);
    GOD_LAUNCH(root_grad_partial, kGradBlocks, kGradThreads, 0, st, theta.p, xs.p, ys.p, S, inv_n, partial.p);
    GOD_LAUNCH(root_reduce_adam, 1, 128, 0, st, partial.p, kGradBlocks, gbest.p, nullptr, nullptr, nullptr, 0, 0.0f,
               0, inv_n);
    // 2. Adam on all parameters with the forward/backward kernels (small steps:
    //    the start is already near the optimum)
    for (int it = 1; it <= steps; ++it) {
      const float lr = 1e-7f + 0.5f * (1e-5f - 1e-7f) * (1.0f + cosf(3.14159265f * (float)(it - 1) / (float)steps));
      GOD_LAUNCH(root_grad_partial, kGradBlocks, kGradThreads, 0, st, theta.p, xs.p, ys.p, S, inv_n, partial.p);
      GOD_LAUNCH(root_reduce_adam, 1, 128, 0, st, partial.p, kGradBlocks, gout.p, theta.p, m1.p, m2.p, it, lr, 1,
                 inv_n);
    }
    // final loss at the trained parameters
    GOD_LAUNCH(root_grad_partial, kGradBlocks, kGradThreads, 0, st, theta.p, xs.p, ys.p, S, inv_n, partial.p);
    GOD_LAUNCH(root_reduce_adam, 1, 128, 0, st, partial.p, kGradBlocks, gout.p, nullptr, nullptr, nullptr, 0, 0.0f, 0,
               inv_n);
    float lsq_loss = 0.0f;
    GOD_CK(cudaMemcpyAsync(&loss, gout.p + NP, sizeof(float), cudaMemcpyDeviceToHost, st));
    GOD_CK(cudaMemcpyAsync(&lsq_loss, gbest.p + NP, sizeof(float), cudaMemcpyDeviceToHost, st));
    GOD_CK(cudaStreamSynchronize(st));
    if (!(loss <= lsq_loss)) {  // keep the better of the two (also when Adam produced NaN)
      loss = lsq_loss;
      GOD_CK(cudaMemcpyAsync(th, best.p, sizeof(th), cudaMemcpyDeviceToHost, st));
    } else {
      GOD_CK(cudaMemcpyAsync(th, theta.p, sizeof(th), cudaMemcpyDeviceToHost, st));
    }
    GOD_CK(cudaStreamSynchronize(st));
    for (int h = 0; h < H; ++h) { R.W1[h] = th[h]; R.b1[h] = th[H + h]; R.W2[h] = th[2 * H + h]; }
    R.b2 = th[3 * H];
  }
  rmi_root_pieces(R);
  GOD_CK(cudaMemcpyAsync(d_root.p, &R, sizeof(R), cudaMemcpyHostToDevice, st));

  // route every key, group by leaf (stable: ranks stay ascending), fit leaves
  DBuf<uint64_t> lk, rv;
  DBuf<uint32_t> lo, hi;
  DBuf<RmiLeaf> leaves;
  DBuf<unsigned long long> stats;
  GOD_TRY(lk.alloc(U, st));
  GOD_TRY(rv.alloc(U, st));
  GOD_TRY(lo.alloc(n_leaves, st));
  GOD_TRY(hi.alloc(n_leaves, st));
  GOD_TRY(leaves.alloc(n_leaves, st));
  GOD_TRY(stats.alloc(8, st));
  const unsigned g = (unsigned)std::min<uint64_t>((U + 255) / 256, (uint64_t)num_sms() * 32);
  GOD_LAUNCH(route_keys, g, 256, 0, st, d_root.p, idx->d_keys, U, lk.p, rv.p);
  // Keys of a leaf are contiguous in rank order when the routing is monotone
  // (the usual case); only otherwise group them by leaf with a sort.
  DBuf<int> nonmono;
  GOD_TRY(nonmono.alloc(1, st));
  GOD_CK(cudaMemsetAsync(nonmono.p, 0, sizeof(int), st));
  GOD_LAUNCH(leaf_monotone, g, 256, 0, st, lk.p, U, nonmono.p);
  int h_nonmono = 0;
  GOD_CK(cudaMemcpyAsync(&h_nonmono, nonmono.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  if (h_nonmono) GOD_TRY(radix_sort_pairs(lk.p, rv.p, U, bits, st));
  GOD_CK(cudaMemsetAsync(lo.p, 0, n_leaves * sizeof(uint32_t), st));
  GOD_CK(cudaMemsetAsync(hi.p, 0, n_leaves * sizeof(uint32_t), st));
  GOD_CK(cudaMemsetAsync(stats.p, 0, 8 * sizeof(unsigned long long), st));
  GOD_LAUNCH(leaf_bounds, g, 256, 0, st, lk.p, U, lo.p, hi.p);
  const unsigned gl = (unsigned)std::min<uint64_t>(((uint64_t)n_leaves + 255) / 256, (uint64_t)num_sms() * 32);
  GOD_LAUNCH(fit_leaves, gl, 256, 0, st, idx->d_keys, rv.p, lo.p, hi.p, n_leaves, leaves.p, stats.p);
  GOD_LAUNCH(leaf_stats, (unsigned)std::min<uint64_t>((n_leaves + 255) / 256, 4096), 256, 0, st, leaves.p, lo.p, hi.p,
             n_leaves, idx->params.rmi_eps_max, stats.p);
  unsigned long long hs[8];
  GOD_CK(cudaMemcpyAsync(hs, stats.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  idx->root = R;
  idx->d_root = d_root.take();
  idx->d_leaves = leaves.take();
  idx->has_rmi = 1;
  idx->rmi_mean_eps = (double)hs[0] / (double)U;
  idx->rmi_fallback_leaves = (uint32_t)hs[3];
  idx->rmi_fallback_key_frac = (double)hs[4] / (double)U;
  idx->rmi_max_eps = (uint32_t)hs[5];
  idx->rmi_loss = loss;
  idx->device_bytes += (uint64_t)n_leaves * sizeof(RmiLeaf) + sizeof(RmiRoot);
  return GOD_OK;
}

}  // namespace god
