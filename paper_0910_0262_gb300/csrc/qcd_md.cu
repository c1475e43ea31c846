// Molecular-dynamics kernels of the hybrid R algorithm (the update the paper's application runs,
// Sec. 1, su3_rmd): Wilson gauge force, plaquette sum, momentum norm and the link update
// U <- exp(eps P) U with reunitarisation; and the per-trajectory measurements (Polyakov loop, the
// dot products of the psi-bar psi estimate).  All FP64.
//
//   S_g = beta sum_x sum_{mu<nu} (1 - Re tr P_{mu nu}(x) / 3)
//   P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
//
// For the link U = U_lambda(x), the plaquettes through it add up to Re tr(U A) with the staple sum
//   A = sum_{nu != lambda} [ U_nu(x+l) U_l(x+nu)^dag U_nu(x)^dag + U_nu(x+l-nu)^dag U_l(x-nu)^dag U_nu(x-nu) ],
// so the Wirtinger gradient is G = -(beta/3) A^dag and the Lie-algebra force (U -> exp(i eps_a T_a) U)
// F = -1/2 P_TA(U G^dag) = (beta/6) P_TA(U A).
#include "qcd_kernels.h"
#include "qcd_su3.cuh"

namespace qcd {

QCD_DEBUG_TAKE(debug_take_md)

namespace {

constexpr int MB = 128;

// traceless anti-Hermitian part (M - M^dag)/2 - tr(M - M^dag)/6
__device__ __forceinline__ M3 project_ta(const M3& m) {
  M3 r;
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const C d = m.e[3 * a + b] - conj(m.e[3 * b + a]);
      r.e[3 * a + b] = cmk(0.5 * d.re, 0.5 * d.im);
    }
  const double ti = (r.e[0].im + r.e[4].im + r.e[8].im) / 3.0;
#pragma unroll
  for (int a = 0; a < 3; a++) r.e[4 * a].im -= ti;
  return r;
}

__device__ __forceinline__ M3 load_canon(const double2* U, size_t link) {
  M3 m;
  const double2* q = U + link * 9;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    const double2 v = q[k];
    m.e[k] = cmk(v.x, v.y);
  }
  return m;
}

__device__ __forceinline__ void store_canon(double2* U, size_t link, const M3& m) {
  double2* q = U + link * 9;
#pragma unroll
  for (int k = 0; k < 9; k++) q[k] = make_double2(m.e[k].re, m.e[k].im);
}

// one thread per link (lambda, lexicographic site i): G, or F, into out (canonical), or added to it
__global__ void __launch_bounds__(MB) gauge_force_kernel(Geom g, double beta, const double2* g64, double2* out,
                                                         int gradient, int accumulate) {
  const int V = 2 * g.Vh;
  const long long tid = (long long)blockIdx.x * MB + threadIdx.x;
  if (tid >= 4LL * V) return;
  const int lam = (int)(tid / V), i = (int)(tid - (long long)lam * V);
  int c[4];
  lattice_coords(g, i, c);
  auto at = [&](int dl, int dn, int nu, int dir) {
    int q[4] = {c[0], c[1], c[2], c[3]};
    q[lam] += dl;
    q[nu] += dn;
    return link_at(g, g64, q[0], q[1], q[2], q[3], dir);
  };
  M3 A;
#pragma unroll
  for (int k = 0; k < 9; k++) A.e[k] = cmk(0.0, 0.0);
#pragma unroll
  for (int nu = 0; nu < 4; nu++) {
    if (nu == lam) continue;
    // U_nu(x+l) (U_nu(x) U_l(x+nu))^dag
    const M3 up = mul_nd(at(1, 0, nu, nu), mul(at(0, 0, nu, nu), at(0, 1, nu, lam)));
    // (U_l(x-nu) U_nu(x+l-nu))^dag U_nu(x-nu)
    const M3 dn = mul_dn(mul(at(0, -1, nu, lam), at(1, -1, nu, nu)), at(0, -1, nu, nu));
    A = m3_add(A, m3_add(up, dn));
  }
  M3 res;
  if (gradient) {
    const double f = -beta / 3.0;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) {
        const C v = conj(A.e[3 * b + a]);
        res.e[3 * a + b] = cmk(f * v.re, f * v.im);
      }
  } else {
    const M3 t = project_ta(mul(link_at(g, g64, c[0], c[1], c[2], c[3], lam), A));
    const double f = beta / 6.0;
#pragma unroll
    for (int k = 0; k < 9; k++) res.e[k] = cmk(f * t.e[k].re, f * t.e[k].im);
  }
  const size_t link = (size_t)i * 4 + lam;
  if (accumulate) res = m3_add(res, load_canon(out, link));
  store_canon(out, link, res);
}

// sum over sites and the six planes of Re tr P_{mu nu}(x) / 3
__global__ void __launch_bounds__(MB) plaquette_kernel(Geom g, const double2* g64, ReduceArgs red) {
  const int V = 2 * g.Vh;
  const int i = blockIdx.x * MB + threadIdx.x;
  double v = 0.0;
  if (i < V) {
    int c[4];
    lattice_coords(g, i, c);
#pragma unroll
    for (int mu = 0; mu < 3; mu++)
#pragma unroll
      for (int nu = mu + 1; nu < 4; nu++) {
        int xm[4] = {c[0], c[1], c[2], c[3]}, xn[4] = {c[0], c[1], c[2], c[3]};
        xm[mu] += 1;
        xn[nu] += 1;
        // Re tr(U_mu(x) U_nu(x+mu) (U_nu(x) U_mu(x+nu))^dag)
        const M3 a = mul(link_at(g, g64, c[0], c[1], c[2], c[3], mu), link_at(g, g64, xm[0], xm[1], xm[2], xm[3], nu));
        const M3 b = mul(link_at(g, g64, c[0], c[1], c[2], c[3], nu), link_at(g, g64, xn[0], xn[1], xn[2], xn[3], mu));
        double tr = 0.0;
#pragma unroll
        for (int k = 0; k < 9; k++) tr += a.e[k].re * b.e[k].re + a.e[k].im * b.e[k].im;  // Re tr(a b^dag)
        v += tr / 3.0;
      }
  }
  block_partial<MB>(v, 0, blockIdx.x, gridDim.x, red);
  grid_finish<MB>(1, gridDim.x, gridDim.x, red);
}

// sum of |z|^2 over n complex numbers
__global__ void __launch_bounds__(MB) flat_norm2_kernel(size_t n, const double2* v, ReduceArgs red) {
  const size_t j = (size_t)blockIdx.x * MB + threadIdx.x;
  double s = 0.0;
  if (j < n) {
    const double2 z = v[j];
    s = z.x * z.x + z.y * z.y;
  }
  block_partial<MB>(s, 0, blockIdx.x, gridDim.x, red);
  grid_finish<MB>(1, gridDim.x, gridDim.x, red);
}

// Polyakov loop: per spatial site, tr prod_t U_t(x, t) / 3; real and imaginary parts summed as RHS
// 0 and 1 of the reduction
__global__ void __launch_bounds__(MB) polyakov_kernel(Geom g, const double2* g64, ReduceArgs red) {
  const int XYZ = g.XYZ;
  const int j = blockIdx.x * MB + threadIdx.x;
  C tr = cmk(0.0, 0.0);
  if (j < XYZ) {
    const int q1 = g.dX.div(j);
    const int x = j - q1 * g.X;
    const int z = g.dY.div(q1);
    const int y = q1 - z * g.Y;
    M3 p = link_at(g, g64, x, y, z, 0, 3);
    for (int t = 1; t < g.T; t++) p = mul(p, link_at(g, g64, x, y, z, t, 3));
    tr = p.e[0] + p.e[4] + p.e[8];
  }
  block_partial<MB>(tr.re / 3.0, 0, blockIdx.x, gridDim.x, red);
  block_partial<MB>(tr.im / 3.0, 1, blockIdx.x, gridDim.x, red);
  grid_finish<MB>(2, gridDim.x, gridDim.x, red);
}

// per RHS r (blockIdx.y): Re sum_j conj(a_j) b_j over n complex numbers at offset r * n
__global__ void __launch_bounds__(MB) flat_redot_kernel(size_t n, int nrhs, const double2* a, const double2* b,
                                                        ReduceArgs red) {
  const size_t j = (size_t)blockIdx.x * MB + threadIdx.x;
  const int r = blockIdx.y;
  double s = 0.0;
  if (j < n) {
    const double2 u = a[(size_t)r * n + j], v = b[(size_t)r * n + j];
    s = u.x * v.x + u.y * v.y;
  }
  block_partial<MB>(s, r, blockIdx.x, gridDim.x, red);
  grid_finish<MB>(nrhs, (long long)gridDim.x * gridDim.y, gridDim.x, red);
}

// exp(M) for a 3x3 complex M: scaling by 2^-s until the Frobenius norm r is <= 1/4, the Taylor
// series to the lowest order n with r^(n+1)/(n+1)! <= 1e-17 (at most 12 at r = 1/4; about 8 for the
// eps |P| of a molecular-dynamics step), then s squarings (Moler and Van Loan, "Nineteen dubious ways
// to compute the exponential of a matrix", 2003).  The truncated series is summed in the basis
// I, M, M^2: by the Cayley-Hamilton theorem M^3 = tr(M) M^2 - c M + det(M) I with
// c = (tr(M)^2 - tr(M^2)) / 2, so M^k / k! = a_k I + b_k M + c_k M^2 with
//   (a, b, c)_{k+1} = (c_k det M, a_k - c_k c, b_k + c_k tr M) / (k + 1),
// the same sum as the matrix series, for one matrix product (M^2) instead of one per term.
__device__ M3 expm3(M3 m) {
  double nrm = 0.0;
#pragma unroll
  for (int k = 0; k < 9; k++) nrm += norm2(m.e[k]);
  nrm = sqrt(nrm);
  int s = 0;
  while (nrm > 0.25 && s < 60) {
    nrm *= 0.5;
    s++;
  }
  const double sc = ldexp(1.0, -s);
#pragma unroll
  for (int k = 0; k < 9; k++) m.e[k] = cmk(sc * m.e[k].re, sc * m.e[k].im);
  int order = 0;
  for (double t = 1.0; order < 20; order++) {
    t *= nrm / (order + 1);  // r^(order+1) / (order+1)!
    if (t <= 1e-17) break;
  }
  const M3 m2 = mul(m, m);
  const C tr1 = m.e[0] + m.e[4] + m.e[8];
  const C tr2 = m2.e[0] + m2.e[4] + m2.e[8];
  const C cc = 0.5 * (tr1 * tr1 - tr2);
  const C det = m.e[0] * (m.e[4] * m.e[8] - m.e[5] * m.e[7]) - m.e[1] * (m.e[3] * m.e[8] - m.e[5] * m.e[6]) +
                m.e[2] * (m.e[3] * m.e[7] - m.e[4] * m.e[6]);
  C a = cmk(1.0, 0.0), b = cmk(0.0, 0.0), c = cmk(0.0, 0.0);  // M^k / k! in the basis I, M, M^2
  C sa = a, sb = b, scm = c;                                    // their sums over k <= order
  for (int k = 0; k < order; k++) {
    const double f = 1.0 / (k + 1);
    const C na = f * (c * det), nb = f * (a - c * cc), nc = f * (b + c * tr1);
    a = na;
    b = nb;
    c = nc;
    sa = sa + a;
    sb = sb + b;
    scm = scm + c;
  }
  M3 e;
#pragma unroll
  for (int k = 0; k < 9; k++) e.e[k] = sb * m.e[k] + scm * m2.e[k];
  e.e[0] = e.e[0] + sa;
  e.e[4] = e.e[4] + sa;
  e.e[8] = e.e[8] + sa;
  for (int k = 0; k < s; k++) e = mul(e, e);
  return e;
}

// rows 0 and 1 orthonormalised (Gram-Schmidt), row 2 = conj(row 0 x row 1)
__device__ __forceinline__ M3 reunitarise(M3 u) {
  double n0 = 0.0;
#pragma unroll
  for (int j = 0; j < 3; j++) n0 += norm2(u.e[j]);
  const double i0 = 1.0 / sqrt(n0);
#pragma unroll
  for (int j = 0; j < 3; j++) u.e[j] = cmk(i0 * u.e[j].re, i0 * u.e[j].im);
  C d = cmk(0.0, 0.0);  // <row 0, row 1>
#pragma unroll
  for (int j = 0; j < 3; j++) d = cfmac(u.e[j], u.e[3 + j], d);
#pragma unroll
  for (int j = 0; j < 3; j++) u.e[3 + j] = u.e[3 + j] - d * u.e[j];
  double n1 = 0.0;
#pragma unroll
  for (int j = 0; j < 3; j++) n1 += norm2(u.e[3 + j]);
  const double i1 = 1.0 / sqrt(n1);
#pragma unroll
  for (int j = 0; j < 3; j++) u.e[3 + j] = cmk(i1 * u.e[3 + j].re, i1 * u.e[3 + j].im);
  u.e[6] = conj(u.e[1] * u.e[5] - u.e[2] * u.e[4]);
  u.e[7] = conj(u.e[2] * u.e[3] - u.e[0] * u.e[5]);
  u.e[8] = conj(u.e[0] * u.e[4] - u.e[1] * u.e[3]);
  return u;
}

// U <- reunitarise(exp(eps P) U) for every link of the canonical fields
__global__ void __launch_bounds__(MB) link_update_kernel(size_t nlinks, double eps, const double2* P, double2* U) {
  const size_t l = (size_t)blockIdx.x * MB + threadIdx.x;
  if (l >= nlinks) return;
  M3 p = load_canon(P, l);
#pragma unroll
  for (int k = 0; k < 9; k++) p.e[k] = cmk(eps * p.e[k].re, eps * p.e[k].im);
  store_canon(U, l, reunitarise(mul(expm3(p), load_canon(U, l))));
}

}  // namespace

void launch_gauge_force(const Geom& g, double beta, const void* g64, double2* out, bool gradient, bool accumulate,
                        cudaStream_t st) {
  g_kernel_launches += 1;
  const long long n = 8LL * g.Vh;
  gauge_force_kernel<<<(unsigned)((n + MB - 1) / MB), MB, 0, st>>>(g, beta, static_cast<const double2*>(g64), out,
                                                                   gradient ? 1 : 0, accumulate ? 1 : 0);
}

void launch_plaquette(const Geom& g, const void* g64, const ReduceArgs& red, cudaStream_t st) {
  g_kernel_launches += 1;
  plaquette_kernel<<<(2 * g.Vh + MB - 1) / MB, MB, 0, st>>>(g, static_cast<const double2*>(g64), red);
}

void launch_flat_norm2(size_t n, const double2* v, const ReduceArgs& red, cudaStream_t st) {
  g_kernel_launches += 1;
  flat_norm2_kernel<<<(unsigned)((n + MB - 1) / MB), MB, 0, st>>>(n, v, red);
}

void launch_polyakov(const Geom& g, const void* g64, const ReduceArgs& red, cudaStream_t st) {
  g_kernel_launches += 1;
  polyakov_kernel<<<(g.XYZ + MB - 1) / MB, MB, 0, st>>>(g, static_cast<const double2*>(g64), red);
}

void launch_flat_redot(size_t n, int nrhs, const double2* a, const double2* b, const ReduceArgs& red,
                       cudaStream_t st) {
  g_kernel_launches += 1;
  flat_redot_kernel<<<dim3((unsigned)((n + MB - 1) / MB), nrhs), MB, 0, st>>>(n, nrhs, a, b, red);
}

void launch_link_update(size_t nlinks, double eps, const double2* P, double2* U, cudaStream_t st) {
  g_kernel_launches += 1;
  link_update_kernel<<<(unsigned)((nlinks + MB - 1) / MB), MB, 0, st>>>(nlinks, eps, P, U);
}

}  // namespace qcd
