// Divide-and-conquer eigensolver for a symmetric tridiagonal matrix (Cuppen's
// method with the eigenvector formula of Gu and Eisenstat), all in FP64.
//
// Tearing: every off-diagonal e_k is removed with a rank-one term
// |e_k| w w^T, w = u_k + sign(e_k) u_{k+1}, so the leaves are 1 x 1 blocks
// with diagonal d_i - |e_{i-1}| - |e_i| and identity eigenvectors.  Level l
// merges neighbouring blocks of size 2^{l-1}:
//
//   diag(Q1, Q2)^T T diag(Q1, Q2) = D + rho z z^T,
//   z = [last row of Q1, sign(e) first row of Q2] / sqrt(2),  rho = 2 |e|.
//
// Per merge: sort the poles, deflate (tiny rho z_i, or two poles closer than
// the tolerance, removed by a Givens rotation), solve the secular equation
//   f(lambda) = 1 + rho sum_j z_j^2 / (d_j - lambda) = 0
// for every root by bisection in the shifted variable mu = lambda - d_origin
// (origin = the nearer pole, so lambda - d_j is formed without cancellation),
// recompute z from the roots (Gu-Eisenstat: z_i^2 = prod_j (lambda_j - d_i) /
// (rho prod_{j != i} (d_j - d_i))) so that the eigenvectors
// v_j = (z_i / (d_i - lambda_j))_i are numerically orthogonal, and multiply the
// permuted/rotated block eigenvectors by the small eigenvector matrix.  Each
// level ends with the block's eigenvalues sorted ascending.

#include <cmath>

#include "ec_sytrd.h"

namespace ec {

struct DcWork {
  int64_t n = 0;
  int* perm = nullptr;
  double* Ds = nullptr;
  double* zs = nullptr;
  double* dtmp = nullptr;
  double* ztmp = nullptr;
  int* defl = nullptr;
  int* ndpos = nullptr;
  int* cmp = nullptr;
  double* dnd = nullptr;
  double* znd = nullptr;
  int* orig = nullptr;
  double* mu = nullptr;
  double* zhat = nullptr;
  int* rank = nullptr;
  int* rot_a = nullptr;
  int* rot_b = nullptr;
  double* rot_c = nullptr;
  double* rot_s = nullptr;
  int* kp = nullptr;
  double* rho = nullptr;
  int* nrot = nullptr;
};

namespace {

constexpr double EPS = 2.220446049250313e-16;

__global__ void leaf_kernel(int64_t n, const double* d, const double* e, double* lam, double* Q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = d[i];
    if (i > 0) v -= fabs(e[i - 1]);
    if (i + 1 < n) v -= fabs(e[i]);
    lam[i] = v;
    Q[i + i * n] = 1.0;
  }
}

// One CTA per merge: gather z, sort the poles, normalise, deflate.
__global__ void __launch_bounds__(256) deflate_kernel(int64_t n, int64_t bs, const double* e,
                                                      const double* lam, const double* Q,
                                                      DcWork w) {
  const int64_t z = blockIdx.x;
  const int64_t s = z * bs, half = bs / 2;
  const int64_t nb = (n - s) < bs ? (n - s) : bs;
  const int64_t nL = half;
  const double er = e[s + half - 1];
  const double sg = er >= 0.0 ? 1.0 : -1.0;
  for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
    w.dtmp[s + i] = lam[s + i];
    w.ztmp[s + i] = (i < nL) ? Q[(s + nL - 1) + (s + i) * n] : sg * Q[(s + nL) + (s + i) * n];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double* D = w.dtmp + s;
  const double* Z = w.ztmp + s;
  int* perm = w.perm + s;
  double* Ds = w.Ds + s;
  double* zs = w.zs + s;
  // merge of two ascending lists
  int64_t a = 0, b = nL;
  for (int64_t p = 0; p < nb; ++p) {
    int64_t idx;
    if (b >= nb || (a < nL && D[a] <= D[b])) idx = a++;
    else idx = b++;
    perm[p] = (int)idx;
    Ds[p] = D[idx];
    zs[p] = Z[idx];
  }
  double zz = 0.0, dmax = 0.0;
  for (int64_t p = 0; p < nb; ++p) {
    zz = fma(zs[p], zs[p], zz);
    dmax = fmax(dmax, fabs(Ds[p]));
  }
  double rho = fabs(er) * zz;
  const double rz = zz > 0.0 ? 1.0 / sqrt(zz) : 0.0;
  for (int64_t p = 0; p < nb; ++p) zs[p] *= rz;
  const double tol = 8.0 * EPS * fmax(dmax, rho);
  int* defl = w.defl + s;
  int* ndpos = w.ndpos + s;
  int* cmp = w.cmp + s;
  int nrot = 0, kp = 0;
  int64_t prev = -1;
  for (int64_t p = 0; p < nb; ++p) {
    cmp[p] = -1;
    if (rho * fabs(zs[p]) <= tol) {
      defl[p] = 1;
      continue;
    }
    if (prev >= 0) {
      const double r = hypot(zs[prev], zs[p]);
      const double c = zs[p] / r, sn = zs[prev] / r;
      if (fabs((Ds[p] - Ds[prev]) * c * sn) <= tol) {
        w.rot_a[s + nrot] = (int)prev;
        w.rot_b[s + nrot] = (int)p;
        w.rot_c[s + nrot] = c;
        w.rot_s[s + nrot] = sn;
        ++nrot;
        const double dp = Ds[prev], dq = Ds[p];
        Ds[prev] = c * c * dp + sn * sn * dq;
        Ds[p] = sn * sn * dp + c * c * dq;
        zs[prev] = 0.0;
        zs[p] = r;
        defl[prev] = 1;
        prev = p;
        continue;
      }
      defl[prev] = 0;
      cmp[prev] = kp;
      ndpos[kp] = (int)prev;
      w.dnd[s + kp] = Ds[prev];
      w.znd[s + kp] = zs[prev];
      ++kp;
    }
    prev = p;
  }
  if (prev >= 0) {
    defl[prev] = 0;
    cmp[prev] = kp;
    ndpos[kp] = (int)prev;
    w.dnd[s + kp] = Ds[prev];
    w.znd[s + kp] = zs[prev];
    ++kp;
  }
  w.kp[z] = kp;
  w.rho[z] = rho;
  w.nrot[z] = nrot;
}

constexpr int64_t SECULAR_WARP_MIN = 256;   // merged size from which a warp solves each root

__device__ __forceinline__ double secular(const double* dnd, const double* znd, int k, double rho,
                                          double dro, double mu) {
  double f0 = 0.0, f1 = 0.0;
  int j = 0;
  for (; j + 1 < k; j += 2) {
    f0 += znd[j] * znd[j] / ((dnd[j] - dro) - mu);
    f1 += znd[j + 1] * znd[j + 1] / ((dnd[j + 1] - dro) - mu);
  }
  if (j < k) f0 += znd[j] * znd[j] / ((dnd[j] - dro) - mu);
  return fma(rho, f0 + f1, 1.0);
}

// With the origin pole o removed: h(mu) = (d_o - d_o - mu) f(mu) = w_o - mu (1 + phi(mu)),
// phi = rho sum_{j != o} z_j^2 / (dd_j - mu).  Returns f (for the bracket), h and h'.
__device__ __forceinline__ void secular_h(const double* dnd, const double* znd, int k, int o,
                                          double rho, double mu, double& f, double& h,
                                          double& hp) {
  const double dro = dnd[o];
  double phi = 0.0, dphi = 0.0;
  for (int j = 0; j < k; ++j) {
    if (j == o) continue;
    const double r = 1.0 / ((dnd[j] - dro) - mu);
    const double t = rho * znd[j] * znd[j] * r;
    phi += t;
    dphi = fma(t, r, dphi);
  }
  const double wo = rho * znd[o] * znd[o];
  h = wo - mu * (1.0 + phi);
  hp = -(1.0 + phi) - mu * dphi;
  f = 1.0 + phi - wo / mu;
}

// Root i of the secular equation: origin at the nearer pole, then Newton steps on
// h (smooth at the origin pole) kept inside the sign bracket of f, with bisection
// whenever a step leaves the bracket.
__global__ void __launch_bounds__(256) secular_kernel(int64_t bs, DcWork w) {
  const int64_t z = blockIdx.x;
  const int64_t s = z * bs;
  const int k = w.kp[z];
  const int i = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const double rho = w.rho[z];
  const double* dnd = w.dnd + s;
  const double* znd = w.znd + s;
  int o;
  double lo, hi;
  if (i < k - 1) {
    const double mid = 0.5 * (dnd[i + 1] - dnd[i]);
    const double f = secular(dnd, znd, k, rho, dnd[i], mid);
    if (f >= 0.0) { o = i; lo = 0.0; hi = mid; }
    else { o = i + 1; lo = -mid; hi = 0.0; }
  } else {
    o = k - 1;
    lo = 0.0;
    hi = rho;
  }
  double mu = 0.5 * (lo + hi);
  for (int it = 0; it < 400; ++it) {
    double f, h, hp;
    secular_h(dnd, znd, k, o, rho, mu, f, h, hp);
    if (f == 0.0) break;
    if (f > 0.0) hi = mu; else lo = mu;
    double nx = (hp != 0.0) ? mu - h / hp : 0.5 * (lo + hi);
    if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
    const bool done = fabs(nx - mu) <= 2.0 * EPS * fabs(nx) || nx == lo || nx == hi;
    mu = nx;
    if (done) break;
  }
  w.orig[s + i] = o;
  w.mu[s + i] = mu;
}

// The same root search with one warp per root: lanes take the poles j = lane (mod 32)
// and the three sums are reduced with shuffles, so every lane holds the same values
// and the warp takes every branch together.  Used for the large merges, where one
// thread per root leaves most of the GPU idle.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) secular_warp_kernel(int64_t bs, DcWork w) {
  const int64_t z = blockIdx.x;
  const int64_t s = z * bs;
  const int k = w.kp[z];
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= k) return;
  const double rho = w.rho[z];
  const double* dnd = w.dnd + s;
  const double* znd = w.znd + s;
  int o;
  double lo, hi;
  if (i < k - 1) {
    const double mid = 0.5 * (dnd[i + 1] - dnd[i]);
    const double dro = dnd[i];
    double part = 0.0;
    for (int j = lane; j < k; j += 32) part += znd[j] * znd[j] / ((dnd[j] - dro) - mid);
    const double f = fma(rho, warp_sum(part), 1.0);
    if (f >= 0.0) { o = i; lo = 0.0; hi = mid; }
    else { o = i + 1; lo = -mid; hi = 0.0; }
  } else {
    o = k - 1;
    lo = 0.0;
    hi = rho;
  }
  const double dro = dnd[o];
  const double wo = rho * znd[o] * znd[o];
  double mu = 0.5 * (lo + hi);
  for (int it = 0; it < 400; ++it) {
    double phi = 0.0, dphi = 0.0;
    for (int j = lane; j < k; j += 32) {
      if (j == o) continue;
      const double r = 1.0 / ((dnd[j] - dro) - mu);
      const double t = rho * znd[j] * znd[j] * r;
      phi += t;
      dphi = fma(t, r, dphi);
    }
    phi = warp_sum(phi);
    dphi = warp_sum(dphi);
    const double h = wo - mu * (1.0 + phi);
    const double hp = -(1.0 + phi) - mu * dphi;
    const double f = 1.0 + phi - wo / mu;
    if (f == 0.0) break;
    if (f > 0.0) hi = mu; else lo = mu;
    double nx = (hp != 0.0) ? mu - h / hp : 0.5 * (lo + hi);
    if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
    const bool done = fabs(nx - mu) <= 2.0 * EPS * fabs(nx) || nx == lo || nx == hi;
    mu = nx;
    if (done) break;
  }
  if (lane == 0) {
    w.orig[s + i] = o;
    w.mu[s + i] = mu;
  }
}

__device__ __forceinline__ double root_minus_pole(const DcWork& w, int64_t s, int j, double di) {
  return (w.dnd[s + w.orig[s + j]] - di) + w.mu[s + j];
}

__global__ void __launch_bounds__(256) zhat_kernel(int64_t bs, DcWork w) {
  const int64_t z = blockIdx.x;
  const int64_t s = z * bs;
  const int k = w.kp[z];
  const int i = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const double* dnd = w.dnd + s;
  const double di = dnd[i];
  double prod = root_minus_pole(w, s, k - 1, di) / w.rho[z];
  for (int j = 0; j < i; ++j) prod *= root_minus_pole(w, s, j, di) / (dnd[j] - di);
  for (int j = i; j < k - 1; ++j) prod *= root_minus_pole(w, s, j, di) / (dnd[j + 1] - di);
  w.zhat[s + i] = copysign(sqrt(fabs(prod)), w.znd[s + i]);
}

__device__ __forceinline__ double item_value(const DcWork& w, int64_t s, int64_t p) {
  if (w.defl[s + p]) return w.Ds[s + p];
  const int i = w.cmp[s + p];
  return w.dnd[s + w.orig[s + i]] + w.mu[s + i];
}

__global__ void __launch_bounds__(256) rank_kernel(int64_t n, int64_t bs, DcWork w, double* lam) {
  const int64_t z = blockIdx.x;
  const int64_t s = z * bs;
  const int64_t nb = (n - s) < bs ? (n - s) : bs;
  const int64_t p = blockIdx.y * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nb) return;
  const double v = item_value(w, s, p);
  int64_t r = 0;
  for (int64_t q = 0; q < nb; ++q) {
    const double u = item_value(w, s, q);
    r += (u < v) || (u == v && q < p);
  }
  w.rank[s + p] = (int)r;
  lam[s + r] = v;
}

// Column rank(p) of the small eigenvector matrix for item p, written with its rows in
// the children's column order: the entry of sorted item r goes to row perm[r].  With
// the deflation rotations applied afterwards (rot_kernel), the merged eigenvectors are
// diag(Q1, Q2) W, so the product needs only the two diagonal blocks (half the flops
// of multiplying a permuted full block).
__global__ void __launch_bounds__(256) vec_kernel(int64_t n, int64_t bs, DcWork w, double* W) {
  const int64_t z = blockIdx.y;
  const int64_t s = z * bs;
  const int64_t nb = (n - s) < bs ? (n - s) : bs;
  const int64_t p = blockIdx.x;
  if (p >= nb) return;
  __shared__ double sh[33];
  double* col = W + s + (s + w.rank[s + p]) * n;
  const int* perm = w.perm + s;
  if (w.defl[s + p]) {
    for (int64_t r = threadIdx.x; r < nb; r += blockDim.x) col[perm[r]] = (r == p) ? 1.0 : 0.0;
    return;
  }
  const int k = w.kp[z];
  const int i = w.cmp[s + p];
  const double dro = w.dnd[s + w.orig[s + i]];
  const double mu = w.mu[s + i];
  double ss = 0.0;
  for (int q = threadIdx.x; q < k; q += blockDim.x) {
    const double v = w.zhat[s + q] / ((w.dnd[s + q] - dro) - mu);
    ss = fma(v, v, ss);
  }
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0) sh[wi] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int x = 0; x < (int)(blockDim.x >> 5); ++x) t += sh[x];
    sh[32] = 1.0 / sqrt(t);
  }
  __syncthreads();
  const double inv = sh[32];
  for (int64_t r = threadIdx.x; r < nb; r += blockDim.x) {
    const int q = w.cmp[s + r];
    col[perm[r]] = (q >= 0) ? inv * (w.zhat[s + q] / ((w.dnd[s + q] - dro) - mu)) : 0.0;
  }
}

// The deflation rotations act on columns (pa, pb) of the permuted children's vectors:
// col_pa <- c col_pa - s col_pb, col_pb <- s col_pa + c col_pb, in rotation order.
// Moved onto the small matrix they become row operations, applied last rotation
// first: row_pa <- c row_pa + s row_pb, row_pb <- -s row_pa + c row_pb (rows in the
// children's order, i.e. perm[pa], perm[pb]).  One thread per column.
__global__ void __launch_bounds__(256) rot_kernel(int64_t n, int64_t bs, DcWork w, double* W) {
  const int64_t z = blockIdx.y;
  const int64_t s = z * bs;
  const int64_t nb = (n - s) < bs ? (n - s) : bs;
  const int nrot = w.nrot[z];
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (nrot == 0 || c >= nb) return;
  double* col = W + s + (s + c) * n;
  const int* perm = w.perm + s;
  for (int t = nrot - 1; t >= 0; --t) {
    const int64_t ra = perm[w.rot_a[s + t]], rb = perm[w.rot_b[s + t]];
    const double cs = w.rot_c[s + t], sn = w.rot_s[s + t];
    const double x = col[ra], y = col[rb];
    col[ra] = fma(cs, x, sn * y);
    col[rb] = fma(-sn, x, cs * y);
  }
}

}  // namespace

DcWork* dc_alloc(int64_t n, cudaError_t (*alloc)(void**, size_t)) {
  DcWork* w = new DcWork();
  w->n = n;
  const size_t nd = sizeof(double) * (size_t)n, ni = sizeof(int) * (size_t)n;
  const size_t nm = (size_t)(n / 2 + 2);
  bool ok = true;
  auto A = [&](void** p, size_t b) { if (ok && alloc(p, b) != cudaSuccess) ok = false; };
  A((void**)&w->perm, ni); A((void**)&w->Ds, nd); A((void**)&w->zs, nd); A((void**)&w->dtmp, nd);
  A((void**)&w->ztmp, nd); A((void**)&w->defl, ni); A((void**)&w->ndpos, ni); A((void**)&w->cmp, ni);
  A((void**)&w->dnd, nd); A((void**)&w->znd, nd); A((void**)&w->orig, ni); A((void**)&w->mu, nd);
  A((void**)&w->zhat, nd); A((void**)&w->rank, ni); A((void**)&w->rot_a, ni); A((void**)&w->rot_b, ni);
  A((void**)&w->rot_c, nd); A((void**)&w->rot_s, nd); A((void**)&w->kp, sizeof(int) * nm);
  A((void**)&w->rho, sizeof(double) * nm); A((void**)&w->nrot, sizeof(int) * nm);
  if (!ok) {
    dc_free(w);
    return nullptr;
  }
  return w;
}

void dc_free(DcWork* w) {
  if (!w) return;
  void* ps[] = {w->perm, w->Ds, w->zs, w->dtmp, w->ztmp, w->defl, w->ndpos, w->cmp, w->dnd, w->znd,
                w->orig, w->mu, w->zhat, w->rank, w->rot_a, w->rot_b, w->rot_c, w->rot_s, w->kp,
                w->rho, w->nrot};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete w;
}

ec_status dc_solve(cudaStream_t s, int64_t n, const double* d, const double* e, double* lam,
                   double* Q, double* Qtmp, double* W, DcWork* wk, DevStatus* st, OzWork* oz) {
  if (n <= 0) return EC_OK;
  cudaMemsetAsync(Q, 0, sizeof(double) * (size_t)n * n, s);
  leaf_kernel<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, ::ec::counted(s)>>>(
      n, d, e, lam, Q);
  double* cur = Q;      // eigenvectors of the current blocks
  double* nxt = Qtmp;   // the merged blocks' eigenvectors
  for (int64_t bs = 2; bs / 2 < n; bs *= 2) {
    const int64_t half = bs / 2;
    const int64_t groups = (n - half + bs - 1) / bs;   // merges with a non-empty right half
    const unsigned chunks = (unsigned)((bs + 255) / 256);
    deflate_kernel<<<(unsigned)groups, 256, 0, ::ec::counted(s)>>>(n, bs, e, lam, cur, *wk);
    if (bs >= SECULAR_WARP_MIN)
      secular_warp_kernel<<<dim3((unsigned)groups, (unsigned)((bs + 7) / 8)), 256, 0,
                            ::ec::counted(s)>>>(bs, *wk);
    else
      secular_kernel<<<dim3((unsigned)groups, chunks), 256, 0, ::ec::counted(s)>>>(bs, *wk);
    zhat_kernel<<<dim3((unsigned)groups, chunks), 256, 0, ::ec::counted(s)>>>(bs, *wk);
    rank_kernel<<<dim3((unsigned)groups, chunks), 256, 0, ::ec::counted(s)>>>(n, bs, *wk, lam);
    vec_kernel<<<dim3((unsigned)bs, (unsigned)groups), 256, 0, ::ec::counted(s)>>>(n, bs, *wk, W);
    rot_kernel<<<dim3(chunks, (unsigned)groups), 256, 0, ::ec::counted(s)>>>(n, bs, *wk, W);
    if (oz && bs >= DC_TC_MIN) {
      // large merges: the two children's diagonal blocks times the matching rows of W,
      // one product per half on the tensor-core path
      for (int64_t z = 0; z < groups; ++z) {
        const int64_t s0 = z * bs, nb = (n - s0) < bs ? (n - s0) : bs;
        gemm_auto(s, oz, N_, N_, half, nb, half, 1.0, cur + s0 + s0 * n, n, W + s0 + s0 * n, n,
                  0.0, nxt + s0 + s0 * n, n, 0, st);
        const int64_t r0 = s0 + half, mb = nb - half;
        gemm_auto(s, oz, N_, N_, mb, nb, mb, 1.0, cur + r0 + r0 * n, n, W + r0 + s0 * n, n, 0.0,
                  nxt + r0 + s0 * n, n, 0, st);
      }
    } else {
      dgemm_halves(s, n, bs, groups, cur, W, nxt, n, st);
    }
    const int64_t done = groups * bs;
    if (done < n)   // a trailing block without a right half is carried over unmerged
      copy_matrix(s, n - done, n - done, cur + done + done * n, n, nxt + done + done * n, n);
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  if (cur != Q) copy_matrix(s, n, n, cur, n, Q, n);
  return EC_OK;
}

}  // namespace ec
