// Fermion force dS/dU for S = phi^dag (Mhat^dag Mhat)^-1 phi, including the
// derivative of the clover term.
//
// The paper's R algorithm (Sec. 1, su3_rmd) evolves the links with this force;
// the paper gives no formula.  With X = (Mhat^dag Mhat)^-1 phi and Y = Mhat X,
//   dS = -2 Re[W^dag dA X] + 2 kappa^2 Re[Y^dag dD X]
// on full-lattice fields X = (X_e, X_o), Y = (Y_e, Y_o), W = (Y_e, kappa^2 Y_o),
// X_o = A_oo^-1 D_oe X_e, Y_o = A_oo^-1 D_eo^dag Y_e.  Every term has the form
// Re tr(C dP) for a product P of links; G = dS/dRe U + i dS/dIm U collects, for
// P = A U B, (B C A)^dag and, for P = A U^dag B, B C A.
//
// Two kernels, all in FP64:
//  1. clover_coeff: per site and plane, C_{mu nu}(x) = -i (kappa c_sw / 4)(S + S^dag)
//     with S the traceless part of sum_s [sigma_{mu nu} X(x)]_s W(x)_s^dag (summed
//     over right-hand sides).
//  2. edge_insert: per link and plane containing it, the two corner insertions next
//     to the link, E = C(x) U_mu(x) + U_mu(x) C(x+mu).
//  3. link_force: per link, the hopping term and the clover leaves through it.
//     A link l sits in two plaquettes of each of its three planes; each plaquette
//     contributes one leaf at each of its four corners, and every such leaf is a
//     cyclic rotation l s1 s2 s3 of the plaquette.  The four corner terms of one
//     plaquette sum to the staple s1 s2 s3 with the corner's C inserted at each
//     corner:  c0 s1 s2 s3 + s1 c1 s2 s3 + s1 s2 c2 s3 + s1 s2 s3 c3
//            = (c0 s1 + s1 c1) s2 s3 + s1 s2 (c2 s3 + s3 c3),
//     and each bracket is the E of s1 or s3 from kernel 2 (for a link walked
//     backwards, s = U^dag, the bracket is -E^dag because C^dag = -C): four
//     products per plaquette instead of eight.
//     The result is either G or F = -1/2 P_TA(U G^dag).
//  4. det_coeff (optional): the clover determinant term's coefficients, added to C before 2.
#include "qcd_dslash.cuh"
#include "qcd_force.h"
#include "qcd_su3.cuh"

namespace qcd {

QCD_DEBUG_TAKE(debug_take_force)

namespace {

constexpr int FB = 128;

// sigma_{mu nu} X: spin s of the result is coef[s] * X[perm[s]] (DeGrand-Rossi;
// planes in the order xy xz xt yz yt zt; coef code 0: 1, 1: -1, 2: i, 3: -i)
__constant__ int SIG_PERM[6][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {1, 0, 3, 2},
                                   {1, 0, 3, 2}, {1, 0, 3, 2}, {0, 1, 2, 3}};
__constant__ int SIG_COEF[6][4] = {{0, 1, 0, 1}, {3, 2, 3, 2}, {1, 1, 0, 0},
                                   {0, 0, 0, 0}, {3, 2, 2, 3}, {1, 0, 0, 1}};

__device__ __forceinline__ C coef_mul(int code, C v) {
  switch (code) {
    case 0: return v;
    case 1: return -v;
    case 2: return times_i(v);
    default: return times_mi(v);
  }
}

__device__ __forceinline__ void load_spinor64(const double2* f, int Vh, int r, int h, C s[12]) {
  SpinorIO<64>::load(f, nullptr, Vh, r, h, s);
}

__device__ __forceinline__ void store_m3(double2* buf, int plane, size_t V, int i, const M3& m) {
  double2* q = buf + (size_t)plane * 9 * V + i;
#pragma unroll
  for (int k = 0; k < 9; k++) q[(size_t)k * V] = make_double2(m.e[k].re, m.e[k].im);
}

__device__ __forceinline__ M3 load_m3(const double2* buf, int plane, size_t V, int i) {
  const double2* q = buf + (size_t)plane * 9 * V + i;
  M3 m;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    double2 v = __ldg(q + (size_t)k * V);
    m.e[k] = cmk(v.x, v.y);
  }
  return m;
}

__device__ __forceinline__ void lex_coords(const Geom& g, int i, int c[4]) {
  lattice_coords(g, i, c);
}

__device__ __forceinline__ int lex_index(const Geom& g, int x, int y, int z, int t) {
  x = wrap(x, g.X);
  y = wrap(y, g.Y);
  z = wrap(z, g.Z);
  t = wrap(t, g.T);
  return x + g.X * (y + g.Y * (z + g.Z * t));
}

// 1. C_{mu nu}(x) for the 6 planes at every site
__global__ void __launch_bounds__(FB) clover_coeff_kernel(Geom g, double kappa, double csw, int nrhs,
                                                          const double2* Xe, const double2* Xo, const double2* Ye,
                                                          const double2* Yo, double2* Cbuf, int accumulate) {
  const int i = blockIdx.x * FB + threadIdx.x;
  const int V = 2 * g.Vh;
  if (i >= V) return;
  int c[4];
  lex_coords(g, i, c);
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int h = i >> 1;
  const double k2 = kappa * kappa;
  M3 S[6];
#pragma unroll
  for (int pl = 0; pl < 6; pl++)
#pragma unroll
    for (int k = 0; k < 9; k++) S[pl].e[k] = cmk(0.0, 0.0);
  for (int r = 0; r < nrhs; r++) {
    C X[12], W[12];
    load_spinor64(p == 0 ? Xe : Xo, g.Vh, r, h, X);
    load_spinor64(p == 0 ? Ye : Yo, g.Vh, r, h, W);
    if (p == 1) {
#pragma unroll
      for (int k = 0; k < 12; k++) W[k] = k2 * W[k];
    }
#pragma unroll
    for (int pl = 0; pl < 6; pl++) {
#pragma unroll
      for (int s = 0; s < 4; s++) {
        const int ps = SIG_PERM[pl][s], cs = SIG_COEF[pl][s];
#pragma unroll
        for (int a = 0; a < 3; a++) {
          const C v = coef_mul(cs, X[3 * ps + a]);
#pragma unroll
          for (int b = 0; b < 3; b++) S[pl].e[3 * a + b] = cfma(v, conj(W[3 * s + b]), S[pl].e[3 * a + b]);
        }
      }
    }
  }
  const double f = kappa * csw / 4.0;
#pragma unroll
  for (int pl = 0; pl < 6; pl++) {
    const double tr = (S[pl].e[0].re + S[pl].e[4].re + S[pl].e[8].re) / 3.0;
    const double ti = (S[pl].e[0].im + S[pl].e[4].im + S[pl].e[8].im) / 3.0;
    S[pl].e[0] = S[pl].e[0] - cmk(tr, ti);
    S[pl].e[4] = S[pl].e[4] - cmk(tr, ti);
    S[pl].e[8] = S[pl].e[8] - cmk(tr, ti);
    M3 Cm;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) {
        const C h2 = S[pl].e[3 * a + b] + conj(S[pl].e[3 * b + a]);
        Cm.e[3 * a + b] = cmk(f * h2.im, -f * h2.re);  // -i f h2
      }
    if (accumulate) Cm = m3_add(Cm, load_m3(Cbuf, pl, V, i));
    store_m3(Cbuf, pl, V, i, Cm);
  }
}

__device__ __forceinline__ void plane_dirs(int pl, int& mu, int& nu) {
  const int M[6] = {0, 0, 0, 1, 1, 2}, N[6] = {1, 2, 3, 2, 3, 3};
  mu = M[pl];
  nu = N[pl];
}

// sum_s v_s w_s^dag over four spins: M[a][b] = sum_s v[s][a] conj(w[s][b])
__device__ __forceinline__ void outer_acc(const C v[12], const C w[12], double scale, M3& m) {
#pragma unroll
  for (int s = 0; s < 4; s++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const C va = scale * v[3 * s + a];
#pragma unroll
      for (int b = 0; b < 3; b++) m.e[3 * a + b] = cfma(va, conj(w[3 * s + b]), m.e[3 * a + b]);
    }
}

// (1 + sgn g_mu) v as a full four-spinor
template <int MU, int SGN>
__device__ __forceinline__ void spin_project_full(const C v[12], C out[12]) {
  C h[6];
  project<MU, SGN>(v, h);
  accumulate<MU, SGN, true>(h, out);
}

template <int MU>
__device__ __forceinline__ void hop_terms(const C Xy[12], const C Yy[12], const C Xn[12], const C Yn[12],
                                          double scale, M3& A, M3& B) {
  C v[12];
  spin_project_full<MU, -1>(Xn, v);  // (1 - g) X(y+mu)
  outer_acc(v, Yy, scale, A);        // G += A^dag
  spin_project_full<MU, +1>(Xy, v);  // (1 + g) X(y)
  outer_acc(v, Yn, scale, B);        // G += B
}

// 3. the clover determinant term S_det = -2 sum_{x odd} log det A(x) of the even-odd preconditioned
// action: dS_det = -2 sum tr(A^-1 dA), and with dA = -kappa c_sw sum sigma_{mu nu} (x) dF_{mu nu} and
// F the traceless part of (Q - Q^dag)/(8i), its leaf coefficient at an odd site is
//   C_{mu nu} = -i (kappa c_sw / 4)(B + B^dag),  B the traceless part of
//   B_ac = sum_t sigma_{mu nu}[t][s] (A^-1)_{(s a),(t c)}  (s = the one spin sigma couples to t),
// the same form as the pseudofermion's clover coefficient; it is added to Cbuf.  One thread per odd
// site reads the two 6x6 blocks of A_oo^-1 (diagonal, then strictly-lower entries).
__global__ void __launch_bounds__(FB) det_coeff_kernel(Geom g, double kappa, double csw, const double2* Ainv_odd,
                                                       double2* Cbuf) {
  const int h = blockIdx.x * FB + threadIdx.x;
  if (h >= g.Vh) return;
  const int V = 2 * g.Vh;
  const Site st = site_of(g, 1, h);
  double d[2][6];
  C L[2][15];
#pragma unroll
  for (int b = 0; b < 2; b++) {
    const double2* q = Ainv_odd + (size_t)(b * 18) * g.Vh + h;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const double2 v = __ldg(q + (size_t)k * g.Vh);
      d[b][2 * k] = v.x;
      d[b][2 * k + 1] = v.y;
    }
#pragma unroll
    for (int k = 0; k < 15; k++) {
      const double2 v = __ldg(q + (size_t)(3 + k) * g.Vh);
      L[b][k] = cmk(v.x, v.y);
    }
  }
  // (A^-1)_{(s a),(t c)} for spins s, t of one chiral block
  auto el = [&](int s, int a, int t, int c) -> C {
    const int b = s >> 1, i6 = 3 * (s & 1) + a, j6 = 3 * (t & 1) + c;
    if (i6 == j6) return cmk(d[b][i6], 0.0);
    if (i6 > j6) return L[b][i6 * (i6 - 1) / 2 + j6];
    return conj(L[b][j6 * (j6 - 1) / 2 + i6]);
  };
  // sigma_{mu nu}[t][PERM[t]] = coefficient COEF[t] (0: 1, 1: -1, 2: i, 3: -i); planes xy xz xt yz yt zt
  constexpr int PERM[6][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {1, 0, 3, 2}, {1, 0, 3, 2}, {1, 0, 3, 2}, {0, 1, 2, 3}};
  constexpr int COEF[6][4] = {{0, 1, 0, 1}, {3, 2, 3, 2}, {1, 1, 0, 0}, {0, 0, 0, 0}, {3, 2, 2, 3}, {1, 0, 0, 1}};
  const double f = kappa * csw / 4.0;
#pragma unroll
  for (int pl = 0; pl < 6; pl++) {
    M3 B;
#pragma unroll
    for (int k = 0; k < 9; k++) B.e[k] = cmk(0.0, 0.0);
#pragma unroll
    for (int t = 0; t < 4; t++)
#pragma unroll
      for (int a = 0; a < 3; a++)
#pragma unroll
        for (int c = 0; c < 3; c++) B.e[3 * a + c] = B.e[3 * a + c] + coef_mul(COEF[pl][t], el(PERM[pl][t], a, t, c));
    const double tr = (B.e[0].re + B.e[4].re + B.e[8].re) / 3.0;
    const double ti = (B.e[0].im + B.e[4].im + B.e[8].im) / 3.0;
    B.e[0] = B.e[0] - cmk(tr, ti);
    B.e[4] = B.e[4] - cmk(tr, ti);
    B.e[8] = B.e[8] - cmk(tr, ti);
    M3 Cm = load_m3(Cbuf, pl, V, st.i);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const C h2 = B.e[3 * a + c] + conj(B.e[3 * c + a]);
        Cm.e[3 * a + c] = Cm.e[3 * a + c] + cmk(f * h2.im, -f * h2.re);  // -i f h2
      }
    store_m3(Cbuf, pl, V, st.i, Cm);
  }
}

// 2. per site x and plane (mu, nu): E of U_mu(x) into field 2 pl, E of U_nu(x) into field 2 pl + 1
__global__ void __launch_bounds__(FB) edge_insert_kernel(Geom g, const double2* g64, const double2* Cbuf,
                                                         double2* Ebuf) {
  const int V = 2 * g.Vh;
  const long long tid = (long long)blockIdx.x * FB + threadIdx.x;
  if (tid >= 6LL * V) return;
  const int pl = (int)(tid / V), i = (int)(tid - (long long)pl * V);
  int mu, nu;
  plane_dirs(pl, mu, nu);
  int c[4];
  lex_coords(g, i, c);
  const M3 C0 = load_m3(Cbuf, pl, V, i);
  int q[4] = {c[0], c[1], c[2], c[3]};
  q[mu] += 1;
  M3 U = link_at(g, g64, c[0], c[1], c[2], c[3], mu);
  M3 Cn = load_m3(Cbuf, pl, V, lex_index(g, q[0], q[1], q[2], q[3]));
  store_m3(Ebuf, 2 * pl, V, i, m3_add(mul(C0, U), mul(U, Cn)));
  q[mu] -= 1;
  q[nu] += 1;
  U = link_at(g, g64, c[0], c[1], c[2], c[3], nu);
  Cn = load_m3(Cbuf, pl, V, lex_index(g, q[0], q[1], q[2], q[3]));
  store_m3(Ebuf, 2 * pl + 1, V, i, m3_add(mul(C0, U), mul(U, Cn)));
}

__device__ __forceinline__ M3 m3_sub(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int k = 0; k < 9; k++) c.e[k] = a.e[k] - b.e[k];
  return c;
}

// 3. per link (y, lambda): hopping term + the clover leaves through the link
__global__ void __launch_bounds__(FB) link_force_kernel(Geom g, double kappa, int nrhs, const double2* g64,
                                                        const double2* Xe, const double2* Xo, const double2* Ye,
                                                        const double2* Yo, const double2* Ebuf, double2* out,
                                                        int gradient, int with_clover, int accumulate) {
  const int V = 2 * g.Vh;
  const long long tid = (long long)blockIdx.x * FB + threadIdx.x;
  if (tid >= 4LL * V) return;
  const int lam = (int)(tid / V), i = (int)(tid - (long long)lam * V);
  int c[4];
  lex_coords(g, i, c);
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  int cl[4] = {c[0], c[1], c[2], c[3]};
  cl[lam] += 1;
  const int j = lex_index(g, cl[0], cl[1], cl[2], cl[3]);
  // hopping part
  M3 Ah, Bh;
#pragma unroll
  for (int k = 0; k < 9; k++) Ah.e[k] = Bh.e[k] = cmk(0.0, 0.0);
  double sgn = 1.0;
  if (lam == 3 && c[3] == g.T - 1) sgn = g.t_bc;
  const double scale = 2.0 * kappa * kappa * sgn;
  for (int r = 0; r < nrhs; r++) {
    C Xy[12], Yy[12], Xn[12], Yn[12];
    load_spinor64(p == 0 ? Xe : Xo, g.Vh, r, i >> 1, Xy);
    load_spinor64(p == 0 ? Ye : Yo, g.Vh, r, i >> 1, Yy);
    load_spinor64(p == 0 ? Xo : Xe, g.Vh, r, j >> 1, Xn);
    load_spinor64(p == 0 ? Yo : Ye, g.Vh, r, j >> 1, Yn);
    switch (lam) {
      case 0: hop_terms<0>(Xy, Yy, Xn, Yn, scale, Ah, Bh); break;
      case 1: hop_terms<1>(Xy, Yy, Xn, Yn, scale, Ah, Bh); break;
      case 2: hop_terms<2>(Xy, Yy, Xn, Yn, scale, Ah, Bh); break;
      default: hop_terms<3>(Xy, Yy, Xn, Yn, scale, Ah, Bh); break;
    }
  }
  M3 G = m3_add(m3_dag(Ah), Bh);
  // clover part: the two plaquettes of each plane containing lambda, each as E s2 s3 + s1 s2 E'
  auto site_off = [&](int d1, int s1, int d2, int s2) {
    int q[4] = {c[0], c[1], c[2], c[3]};
    q[d1] += s1;
    q[d2] += s2;
    return lex_index(g, q[0], q[1], q[2], q[3]);
  };
  auto link_off = [&](int d1, int s1, int d2, int s2, int dir) {
    int q[4] = {c[0], c[1], c[2], c[3]};
    q[d1] += s1;
    q[d2] += s2;
    return link_at(g, g64, q[0], q[1], q[2], q[3], dir);
  };
  for (int pl = 0; pl < 6 && with_clover; pl++) {
    int mu, nu;
    plane_dirs(pl, mu, nu);
    if (mu != lam && nu != lam) continue;
    if (lam == mu) {
      // E of the nu links of the plane
      auto Eat = [&](int dm, int dn) { return load_m3(Ebuf, 2 * pl + 1, V, site_off(mu, dm, nu, dn)); };
      // plaquette at y: s1 = U_nu(y+mu), s2 = A^dag, s3 = B^dag with A = U_mu(y+nu), B = U_nu(y);
      // T = E_nu(y+mu) s2 s3 - s1 s2 E_nu(y)^dag and G += T^dag = (B A) E_nu(y+mu)^dag - E_nu(y) (A s1^dag)
      {
        const M3 A = link_off(mu, 0, nu, 1, mu), B = link_off(mu, 0, nu, 0, nu), s1 = link_off(mu, 1, nu, 0, nu);
        G = m3_add(G, m3_sub(mul_nd(mul(B, A), Eat(1, 0)), mul(Eat(0, 0), mul_nd(A, s1))));
      }
      // plaquette at y-nu (the link enters daggered): s1 = D^dag, s2 = P, s3 = Q with D = U_nu(y-nu),
      // P = U_mu(y-nu), Q = U_nu(y+mu-nu); G += -E_nu(y-nu)^dag (P Q) + (D^dag P) E_nu(y+mu-nu)
      {
        const M3 D = link_off(mu, 0, nu, -1, nu), P = link_off(mu, 0, nu, -1, mu), Q = link_off(mu, 1, nu, -1, nu);
        G = m3_add(G, m3_sub(mul(mul_dn(D, P), Eat(1, -1)), mul_dn(Eat(0, -1), mul(P, Q))));
      }
    } else {
      // E of the mu links of the plane
      auto Eat = [&](int dm, int dn) { return load_m3(Ebuf, 2 * pl, V, site_off(mu, dm, nu, dn)); };
      // plaquette at y-mu: s1 = A^dag, s2 = B^dag, s3 = S with A = U_mu(y-mu+nu), B = U_nu(y-mu),
      // S = U_mu(y-mu); G += T^dag = -(S^dag B) E_mu(y-mu+nu) + E_mu(y-mu)^dag (B A)
      {
        const M3 A = link_off(mu, -1, nu, 1, mu), B = link_off(mu, -1, nu, 0, nu), S = link_off(mu, -1, nu, 0, mu);
        G = m3_add(G, m3_sub(mul_dn(Eat(-1, 0), mul(B, A)), mul(mul_dn(S, B), Eat(-1, 1))));
      }
      // plaquette at y (the link enters daggered): s1 = S0 = U_mu(y), s2 = R = U_nu(y+mu),
      // s3 = A^dag with A = U_mu(y+nu); G += E_mu(y) (R A^dag) - (S0 R) E_mu(y+nu)^dag
      {
        const M3 S0 = link_off(mu, 0, nu, 0, mu), R = link_off(mu, 1, nu, 0, nu), A = link_off(mu, 0, nu, 1, mu);
        G = m3_add(G, m3_sub(mul(Eat(0, 0), mul_nd(R, A)), mul_nd(mul(S0, R), Eat(0, 1))));
      }
    }
  }
  M3 res;
  if (gradient) {
    res = G;
  } else {
    // F = -1/2 P_TA(U G^dag)
    const M3 U = link_at(g, g64, c[0], c[1], c[2], c[3], lam);
    const M3 M = mul_nd(U, G);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) {
        const C d = M.e[3 * a + b] - conj(M.e[3 * b + a]);
        res.e[3 * a + b] = cmk(-0.25 * d.re, -0.25 * d.im);
      }
    const double ti = (res.e[0].im + res.e[4].im + res.e[8].im) / 3.0;
#pragma unroll
    for (int a = 0; a < 3; a++) res.e[4 * a].im -= ti;
  }
  double2* q = out + ((size_t)i * 4 + lam) * 9;
  if (accumulate) {
#pragma unroll
    for (int k = 0; k < 9; k++) {
      const double2 o = q[k];
      q[k] = make_double2(o.x + res.e[k].re, o.y + res.e[k].im);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 9; k++) q[k] = make_double2(res.e[k].re, res.e[k].im);
  }
}

}  // namespace

size_t force_clover_bytes(const Geom& g) { return (size_t)6 * 9 * 2 * g.Vh * sizeof(double2); }

void launch_force_coeff(const Geom& g, double kappa, double csw, int nrhs, const double2* Xe, const double2* Xo,
                        const double2* Ye, const double2* Yo, double2* Cbuf, bool accumulate, cudaStream_t st) {
  g_kernel_launches += 1;
  const int V = 2 * g.Vh;
  clover_coeff_kernel<<<(V + FB - 1) / FB, FB, 0, st>>>(g, kappa, csw, nrhs, Xe, Xo, Ye, Yo, Cbuf,
                                                        accumulate ? 1 : 0);
}

size_t force_edge_bytes(const Geom& g) { return 2 * force_clover_bytes(g); }

void launch_force_edges(const Geom& g, const void* g64, const double2* Cbuf, double2* Ebuf, cudaStream_t st) {
  g_kernel_launches += 1;
  const int V = 2 * g.Vh;
  edge_insert_kernel<<<(int)((6LL * V + FB - 1) / FB), FB, 0, st>>>(g, static_cast<const double2*>(g64), Cbuf,
                                                                     Ebuf);
}

void launch_force_links(const Geom& g, double kappa, int nrhs, const void* g64, const double2* Xe, const double2* Xo,
                        const double2* Ye, const double2* Yo, const double2* Ebuf, double2* out, bool gradient,
                        bool with_clover, bool accumulate, cudaStream_t st) {
  g_kernel_launches += 1;
  const int V = 2 * g.Vh;
  link_force_kernel<<<(int)((4LL * V + FB - 1) / FB), FB, 0, st>>>(g, kappa, nrhs, static_cast<const double2*>(g64),
                                                                    Xe, Xo, Ye, Yo, Ebuf, out, gradient ? 1 : 0,
                                                                    with_clover ? 1 : 0, accumulate ? 1 : 0);
}

void launch_force_det_coeff(const Geom& g, double kappa, double csw, const double2* Ainv_odd, double2* Cbuf,
                            cudaStream_t st) {
  g_kernel_launches += 1;
  det_coeff_kernel<<<(g.Vh + FB - 1) / FB, FB, 0, st>>>(g, kappa, csw, Ainv_odd, Cbuf);
}

// clover part per link: 6 plaquettes x (4 products of 198 flops + 36 adds); per site of kernel 2:
// 6 planes x 2 links x (2 products + 18 adds)
double force_link_flops(int nrhs, bool with_clover) { return (with_clover ? 6.0 * 828.0 : 0.0) + 744.0 * nrhs + 274.0; }
double force_edge_flops() { return 6.0 * 2 * (2 * 198.0 + 18.0); }
double force_coeff_flops(int nrhs) { return 6.0 * (4 * 3 * 3 * 8.0) * nrhs + 6.0 * 60.0; }

}  // namespace qcd
