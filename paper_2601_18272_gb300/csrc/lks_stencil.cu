// LKS predictor (Sec. 2.2) and its exact transpose on D2Q9, one CTA per 32x8 tile.
//
// Forward, per cell x (tau = 1 so f_i* is f_i^eq streamed from x - c_i):
//   f_i^eq(y) = w_i (3p + 3c.u + 9/2 (c.u)^2 - 3/2 |u|^2 + 2A sum_ab G_ab c_a c_b),
//   G_ab = d_b u_a by the isotropic central stencil sum_j c_jb u_a(y + c_j) / 6,
//   p*(x) = 1/3 sum_i f_i^eq(x - c_i),  u*(x) = sum_i c_i f_i^eq(x - c_i).
// Written per node as f_i = w_i (a + c.b + cx^2 Qxx + cy^2 Qyy + cx cy Qxy) with
//   a = 3p - 3/2|u|^2, b = 3u, Qxx = 9/2 ux^2 + 2A Gxx, Qyy = 9/2 uy^2 + 2A Gyy,
//   Qxy = 9 ux uy + 2A (Gxy + Gyx),
// the six coefficients are computed once per node of the tile + halo 1 in shared memory and
// gathered by the nine neighbours. Boundary values are prescribed directly (Sec. 2.2): walls in
// y (u = 0, p from the inner row) for x-interior nodes, then open x planes (inflow u = u_in and
// p copied inward, outflow p = 0 and u copied inward; pressure-driven p = dp / 0 and u copied).
// Ghosts for the gradient: open planes copy the boundary node, walls reflect u with a sign flip.
//
// Algorithmic traffic per cell: read p, u (3 values), write p*, u* (3 values): 24 B in FP32.
#include "lks_kernels.h"
#include "lks_stencil_common.cuh"

namespace lks {

namespace {

constexpr int TX = kTileX, TY = kTileY2;
constexpr int HX = TX + 4, HY = TY + 4;  // halo-2 region
constexpr int CX = TX + 2, CY = TY + 2;  // halo-1 region

__device__ __forceinline__ bool interior_x(const Geo& g, int x) { return interior_axis(g.bc[0], g.n[0], x); }
__device__ __forceinline__ bool interior_y(const Geo& g, int y) { return interior_axis(g.bc[1], g.n[1], y); }

template <typename T>
__global__ void __launch_bounds__(TX* TY) k_stencil2d(Geo g, Slots<T> S, const Ctrl* __restrict__ ctrl, int di) {
  __shared__ T sp[HY][HX], sux[HY][HX], suy[HY][HX];
  __shared__ T ca[CY][CX], cbx[CY][CX], cby[CY][CX], cqxx[CY][CX], cqyy[CY][CX], cqxy[CY][CX];
  __shared__ T op[TY][TX], oux[TY][TX], ouy[TY][TX];
  const int t = ctrl->t0 + di, base = ctrl->base;
  const T* __restrict__ src = slot_ptr(S, t - 1, base);
  T* __restrict__ dst = slot_ptr(S, t, base);
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;

  for (int q = tid; q < HX * HY; q += TX * TY) {
    const int li = q % HX, lj = q / HX;
    int gx = x0 - 2 + li, gy = y0 - 2 + lj, sgn = 1;
    T p = T(0), ux = T(0), uy = T(0);
    if (ghost_axis(g.bc[0], nx, &gx, &sgn) && ghost_axis(g.bc[1], ny, &gy, &sgn)) {
      const long long n = gx + (long long)nx * gy;
      p = src[n];
      ux = T(sgn) * src[N + n];
      uy = T(sgn) * src[2 * N + n];
    }
    sp[lj][li] = p;
    sux[lj][li] = ux;
    suy[lj][li] = uy;
  }
  __syncthreads();

  const T A2 = two_a<T>(g);
  const T sixth = T(1.0 / 6.0);
  for (int q = tid; q < CX * CY; q += TX * TY) {
    const int ci = q % CX, cj = q / CX, li = ci + 1, lj = cj + 1;
    const T ux = sux[lj][li], uy = suy[lj][li], p = sp[lj][li];
    const T gxx = (sux[lj][li + 1] - sux[lj][li - 1] + sux[lj + 1][li + 1] - sux[lj + 1][li - 1] +
                   sux[lj - 1][li + 1] - sux[lj - 1][li - 1]) * sixth;
    const T gxy = (sux[lj + 1][li] - sux[lj - 1][li] + sux[lj + 1][li + 1] + sux[lj + 1][li - 1] -
                   sux[lj - 1][li + 1] - sux[lj - 1][li - 1]) * sixth;
    const T gyx = (suy[lj][li + 1] - suy[lj][li - 1] + suy[lj + 1][li + 1] - suy[lj + 1][li - 1] +
                   suy[lj - 1][li + 1] - suy[lj - 1][li - 1]) * sixth;
    const T gyy = (suy[lj + 1][li] - suy[lj - 1][li] + suy[lj + 1][li + 1] + suy[lj + 1][li - 1] -
                   suy[lj - 1][li + 1] - suy[lj - 1][li - 1]) * sixth;
    ca[cj][ci] = T(3) * p - T(1.5) * (ux * ux + uy * uy);
    cbx[cj][ci] = T(3) * ux;
    cby[cj][ci] = T(3) * uy;
    cqxx[cj][ci] = T(4.5) * ux * ux + A2 * gxx;
    cqyy[cj][ci] = T(4.5) * uy * uy + A2 * gyy;
    cqxy[cj][ci] = T(9) * ux * uy + A2 * (gxy + gyx);
  }
  __syncthreads();

  const int gx = x0 + tx, gy = y0 + ty;
  const bool ingrid = gx < nx && gy < ny;
  {
    const int ci = tx + 1, cj = ty + 1;
    const T w1 = T(1.0 / 9.0), w5 = T(1.0 / 36.0);
    const T f0 = T(4.0 / 9.0) * ca[cj][ci];
    const T f1 = w1 * (ca[cj][ci - 1] + cbx[cj][ci - 1] + cqxx[cj][ci - 1]);
    const T f2 = w1 * (ca[cj - 1][ci] + cby[cj - 1][ci] + cqyy[cj - 1][ci]);
    const T f3 = w1 * (ca[cj][ci + 1] - cbx[cj][ci + 1] + cqxx[cj][ci + 1]);
    const T f4 = w1 * (ca[cj + 1][ci] - cby[cj + 1][ci] + cqyy[cj + 1][ci]);
    const T f5 = w5 * (ca[cj - 1][ci - 1] + cbx[cj - 1][ci - 1] + cby[cj - 1][ci - 1] + cqxx[cj - 1][ci - 1] +
                       cqyy[cj - 1][ci - 1] + cqxy[cj - 1][ci - 1]);
    const T f6 = w5 * (ca[cj - 1][ci + 1] - cbx[cj - 1][ci + 1] + cby[cj - 1][ci + 1] + cqxx[cj - 1][ci + 1] +
                       cqyy[cj - 1][ci + 1] - cqxy[cj - 1][ci + 1]);
    const T f7 = w5 * (ca[cj + 1][ci + 1] - cbx[cj + 1][ci + 1] - cby[cj + 1][ci + 1] + cqxx[cj + 1][ci + 1] +
                       cqyy[cj + 1][ci + 1] + cqxy[cj + 1][ci + 1]);
    const T f8 = w5 * (ca[cj + 1][ci - 1] + cbx[cj + 1][ci - 1] - cby[cj + 1][ci - 1] + cqxx[cj + 1][ci - 1] +
                       cqyy[cj + 1][ci - 1] - cqxy[cj + 1][ci - 1]);
    op[ty][tx] = (f0 + f1 + f2 + f3 + f4 + f5 + f6 + f7 + f8) * T(1.0 / 3.0);
    oux[ty][tx] = f1 - f3 + f5 - f6 - f7 + f8;
    ouy[ty][tx] = f2 - f4 + f5 + f6 - f7 - f8;
  }
  __syncthreads();
  // walls in y, for x-interior nodes
  if (ingrid && g.bc[1] == BC_WALL && (gy == 0 || gy == ny - 1) && interior_x(g, gx)) {
    const int tin = (gy == 0) ? ty + 1 : ty - 1;
    op[ty][tx] = op[tin][tx];
    oux[ty][tx] = T(0);
    ouy[ty][tx] = T(0);
  }
  __syncthreads();
  // open x planes, all rows
  if (ingrid && g.bc[0] != BC_PERIODIC && (gx == 0 || gx == nx - 1)) {
    const bool inlet = gx == 0;
    const int tin = inlet ? tx + 1 : tx - 1;
    if (g.bc[0] == BC_INFLOW_OUTFLOW) {
      if (inlet) {
        op[ty][tx] = op[ty][tin];
        oux[ty][tx] = T(g.u_in);
        ouy[ty][tx] = T(0);
      } else {
        op[ty][tx] = T(0);
        oux[ty][tx] = oux[ty][tin];
        ouy[ty][tx] = ouy[ty][tin];
      }
    } else {
      op[ty][tx] = inlet ? T(g.dp) : T(0);
      oux[ty][tx] = oux[ty][tin];
      ouy[ty][tx] = ouy[ty][tin];
    }
  }
  if (ingrid) {
    const long long n = gx + (long long)nx * gy;
    dst[n] = op[ty][tx];
    dst[N + n] = oux[ty][tx];
    dst[2 * N + n] = ouy[ty][tx];
  }
}

// ---------------------------------------------------------------------------------------------
// Transpose. With fbar_i(z) = 1/3 lam_p*(z + c_i) + c_i . lam_u*(z + c_i) over interior targets
// (after routing the boundary nodes' adjoints back through the boundary rules), per node z:
//   P = sum_i w_i fbar_i, U = sum_i w_i c_i fbar_i, s = sum_i w_i c_i c_i fbar_i,
//   lam_p(z) = 3P,  lam_u(z) = 3U + 9 s u - 3 u P + (2A/6) sum_{(y,j): nbr(y,c_j) = z} sgn c_j . s(y)
// where the last sum is the transpose of the velocity-gradient stencil (with its ghost rule).
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ld_lam(const T* L, long long N, int plane, int x, int y, int nx) {
  return L[plane * N + x + (long long)nx * y];
}

// Adjoint of (p*, u*) seen by interior node (x, y) once the boundary rules are reversed.
template <typename T>
__device__ __forceinline__ void lam_star_adjusted(const Geo& g, const T* L, int x, int y, T* lp, T* lux, T* luy) {
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1];
  if (!interior_x(g, x) || !interior_y(g, y)) {
    *lp = *lux = *luy = T(0);
    return;
  }
  T p = ld_lam(L, N, 0, x, y, nx);
  T ux = ld_lam(L, N, 1, x, y, nx);
  T uy = ld_lam(L, N, 2, x, y, nx);
  const int bx = g.bc[0];
  if (bx == BC_INFLOW_OUTFLOW && x == 1) p += ld_lam(L, N, 0, 0, y, nx);
  if (g.bc[1] == BC_WALL) {
    for (int side = 0; side < 2; ++side) {
      const int yin = side == 0 ? 1 : ny - 2, yw = side == 0 ? 0 : ny - 1;
      if (y != yin) continue;
      p += ld_lam(L, N, 0, x, yw, nx);
      if (bx == BC_INFLOW_OUTFLOW && x == 1) p += ld_lam(L, N, 0, 0, yw, nx);
    }
  }
  if ((bx == BC_INFLOW_OUTFLOW || bx == BC_PRESSURE) && x == nx - 2) {
    ux += ld_lam(L, N, 1, nx - 1, y, nx);
    uy += ld_lam(L, N, 2, nx - 1, y, nx);
  }
  if (bx == BC_PRESSURE && x == 1) {
    ux += ld_lam(L, N, 1, 0, y, nx);
    uy += ld_lam(L, N, 2, 0, y, nx);
  }
  *lp = p;
  *lux = ux;
  *luy = uy;
}

template <typename T>
__global__ void __launch_bounds__(TX* TY) k_stencil2d_adj(Geo g, Slots<T> S, T* Lb, long long lstride,
                                                          const Ctrl* __restrict__ ctrl, int di) {
  __shared__ T lp[HY][HX], lx[HY][HX], ly[HY][HX];
  __shared__ T mP[CY][CX], mUx[CY][CX], mUy[CY][CX], mSxx[CY][CX], mSyy[CY][CX], mSxy[CY][CX];
  const int t = ctrl->t0 - di, base = ctrl->base;
  const T* __restrict__ Lcur = Lb + (long long)(t & 1) * lstride;
  T* __restrict__ Lnext = Lb + (long long)((t - 1) & 1) * lstride;
  const T* __restrict__ st = slot_ptr(S, t - 1, base);
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;

  for (int q = tid; q < HX * HY; q += TX * TY) {
    const int li = q % HX, lj = q / HX;
    int gx = x0 - 2 + li, gy = y0 - 2 + lj;
    T a = T(0), b = T(0), c = T(0);
    bool ok = true;
    if (g.bc[0] == BC_PERIODIC) gx = wrapi(gx, nx);
    else if (gx < 0 || gx >= nx) ok = false;
    if (g.bc[1] == BC_PERIODIC) gy = wrapi(gy, ny);
    else if (gy < 0 || gy >= ny) ok = false;
    if (ok) lam_star_adjusted(g, Lcur, gx, gy, &a, &b, &c);
    lp[lj][li] = a;
    lx[lj][li] = b;
    ly[lj][li] = c;
  }
  __syncthreads();

  const T third = T(1.0 / 3.0), w0 = T(4.0 / 9.0), w1 = T(1.0 / 9.0), w5 = T(1.0 / 36.0);
  for (int q = tid; q < CX * CY; q += TX * TY) {
    const int ci = q % CX, cj = q / CX, li = ci + 1, lj = cj + 1;
    const T f0 = third * lp[lj][li];
    const T f1 = third * lp[lj][li + 1] + lx[lj][li + 1];
    const T f2 = third * lp[lj + 1][li] + ly[lj + 1][li];
    const T f3 = third * lp[lj][li - 1] - lx[lj][li - 1];
    const T f4 = third * lp[lj - 1][li] - ly[lj - 1][li];
    const T f5 = third * lp[lj + 1][li + 1] + lx[lj + 1][li + 1] + ly[lj + 1][li + 1];
    const T f6 = third * lp[lj + 1][li - 1] - lx[lj + 1][li - 1] + ly[lj + 1][li - 1];
    const T f7 = third * lp[lj - 1][li - 1] - lx[lj - 1][li - 1] - ly[lj - 1][li - 1];
    const T f8 = third * lp[lj - 1][li + 1] + lx[lj - 1][li + 1] - ly[lj - 1][li + 1];
    const T d5 = f5 + f6 + f7 + f8;
    mP[cj][ci] = w0 * f0 + w1 * (f1 + f2 + f3 + f4) + w5 * d5;
    mUx[cj][ci] = w1 * (f1 - f3) + w5 * (f5 - f6 - f7 + f8);
    mUy[cj][ci] = w1 * (f2 - f4) + w5 * (f5 + f6 - f7 - f8);
    mSxx[cj][ci] = w1 * (f1 + f3) + w5 * d5;
    mSyy[cj][ci] = w1 * (f2 + f4) + w5 * d5;
    mSxy[cj][ci] = w5 * (f5 - f6 + f7 - f8);
  }
  __syncthreads();

  const int gx = x0 + tx, gy = y0 + ty;
  if (gx < nx && gy < ny) {
    const long long n = gx + (long long)nx * gy;
    const int ci = tx + 1, cj = ty + 1;
    const T ux = st[N + n], uy = st[2 * N + n];
    const T P = mP[cj][ci];
    T gtx, gty;  // sum over (y, j) -> z of sgn * (c_jx s_ax(y) + c_jy s_ay(y))
    const bool near_x = g.bc[0] != BC_PERIODIC && (gx <= 1 || gx >= nx - 2);
    const bool near_y = g.bc[1] != BC_PERIODIC && (gy <= 1 || gy >= ny - 2);
    if (!near_x && !near_y) {
      // interior: y = z - c_j; sum_j c_jx h(z - c_j) = h(W)+h(SW)+h(NW) - h(E)-h(NE)-h(SE)
#define CXS(M) (M[cj][ci - 1] + M[cj - 1][ci - 1] + M[cj + 1][ci - 1] - M[cj][ci + 1] - M[cj + 1][ci + 1] - M[cj - 1][ci + 1])
#define CYS(M) (M[cj - 1][ci] + M[cj - 1][ci - 1] + M[cj - 1][ci + 1] - M[cj + 1][ci] - M[cj + 1][ci + 1] - M[cj + 1][ci - 1])
      gtx = CXS(mSxx) + CYS(mSxy);
      gty = CXS(mSxy) + CYS(mSyy);
#undef CXS
#undef CYS
    } else {
      gtx = gty = T(0);
      const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
      const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int yx = gx + dx, yy = gy + dy;
          if (g.bc[0] == BC_PERIODIC) yx = wrapi(yx, nx);
          else if (yx < 0 || yx >= nx) continue;
          if (g.bc[1] == BC_PERIODIC) yy = wrapi(yy, ny);
          else if (yy < 0 || yy >= ny) continue;
          const T sxx = mSxx[cj + dy][ci + dx], syy = mSyy[cj + dy][ci + dx], sxy = mSxy[cj + dy][ci + dx];
          for (int j = 1; j < 9; ++j) {
            int mx = yx + cx[j], my = yy + cy[j], sgn = 1;
            if (!ghost_axis(g.bc[0], nx, &mx, &sgn) || !ghost_axis(g.bc[1], ny, &my, &sgn)) continue;
            if (mx != gx || my != gy) continue;
            gtx += T(sgn) * (T(cx[j]) * sxx + T(cy[j]) * sxy);
            gty += T(sgn) * (T(cx[j]) * sxy + T(cy[j]) * syy);
          }
        }
    }
    const T kA = two_a<T>(g) * T(1.0 / 6.0);
    Lnext[n] = T(3) * P;
    Lnext[N + n] = T(3) * mUx[cj][ci] + T(9) * (mSxx[cj][ci] * ux + mSxy[cj][ci] * uy) - T(3) * ux * P + kA * gtx;
    Lnext[2 * N + n] = T(3) * mUy[cj][ci] + T(9) * (mSxy[cj][ci] * ux + mSyy[cj][ci] * uy) - T(3) * uy * P + kA * gty;
  }
}

}  // namespace

template <typename T>
void launch_stencil_fwd(const Geo& g, const Slots<T>& S, const Ctrl* ctrl, int di, cudaStream_t st) {
  if (g.dim == 2) {
    dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY);
    k_stencil2d<T><<<grid, dim3(TX, TY), 0, st>>>(g, S, ctrl, di);
  } else {
    launch_stencil3d_fwd<T>(g, S, ctrl, di, st);
  }
}

template <typename T>
void launch_stencil_adj(const Geo& g, const Slots<T>& S, T* Lb, long long lstride, const Ctrl* ctrl, int di,
                        cudaStream_t st) {
  if (g.dim == 2) {
    dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY);
    k_stencil2d_adj<T><<<grid, dim3(TX, TY), 0, st>>>(g, S, Lb, lstride, ctrl, di);
  } else {
    launch_stencil3d_adj<T>(g, S, Lb, lstride, ctrl, di, st);
  }
}

template void launch_stencil_fwd<float>(const Geo&, const Slots<float>&, const Ctrl*, int, cudaStream_t);
template void launch_stencil_fwd<double>(const Geo&, const Slots<double>&, const Ctrl*, int, cudaStream_t);
template void launch_stencil_adj<float>(const Geo&, const Slots<float>&, float*, long long, const Ctrl*, int,
                                        cudaStream_t);
template void launch_stencil_adj<double>(const Geo&, const Slots<double>&, double*, long long, const Ctrl*, int,
                                         cudaStream_t);

}  // namespace lks
