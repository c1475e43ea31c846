// Time decomposition over several GPUs (included once, at the end of qcd_api.cu, whose context and
// helpers it uses).
//
// A t-slab context holds the time slices t_offset .. t_offset + t_local - 1 of a global lattice.  Its
// links, clover term and fields live in the layout of a lattice X x Y x Z x t_local; the extended
// links (two more slices on each side) are kept for the clover build, which runs on the extended
// lattice and keeps the slab's part.  Every hopping pass first packs the input's two t-faces
// (launch_halo_pack), hands them to the caller's exchange callback and then runs the halo variant
// of the split hopping kernel; every CG reduction stores its local total, is summed by the caller's
// allreduce callback and is then finalised on the device with the same code as the single-GPU solve.

namespace {

Geom make_geom(int X, int Y, int Z, int T, double t_bc, int t0, int Tg) {
  Geom g{};
  g.X = X;
  g.Y = Y;
  g.Z = Z;
  g.T = T;
  g.Vh = X * Y * Z * T / 2;
  g.XY = X * Y;
  g.XYZ = X * Y * Z;
  g.t_bc = t_bc;
  g.dX = make_fastdiv(X);
  g.dY = make_fastdiv(Y);
  g.dZ = make_fastdiv(Z);
  g.t0 = t0;
  g.Tg = Tg;
  return g;
}

size_t halo_bytes(const qcd_ctx* c, int prec, int nrhs) {
  return (size_t)(c->g.XYZ / 2) * nrhs * (prec == 64 ? 96 : 48);
}

int recon_of(const qcd_ctx* c, int prec) { return prec == 64 ? 18 : c->recon; }

// the local part of a clover-shaped field [2 parities][rows][Vh_ext] of elements of `elem` bytes: the
// slab's sites start XYZ half indices into each row of the extended lattice (two time slices)
qcd_status copy_slab_rows(qcd_ctx* c, void* dst, const void* src, int rows, size_t elem) {
  const size_t off = (size_t)c->g.XYZ * elem;
  CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)c->g.Vh * elem, static_cast<const char*>(src) + off,
                             (size_t)c->ge.Vh * elem, (size_t)c->g.Vh * elem, (size_t)2 * rows,
                             cudaMemcpyDeviceToDevice, c->st));
  return QCD_OK;
}

qcd_status slab_clover_build(qcd_ctx* c, double kappa, double csw, void* work) {
  const Geom& ge = c->ge;
  if (!c->ext_g64) {
    CUDA_TRY(cudaMalloc(&c->ext_g64, (size_t)2 * 4 * 9 * ge.Vh * sizeof(double2)));
    CUDA_TRY(cudaMalloc(&c->ext_A64, (size_t)2 * 36 * ge.Vh * sizeof(double2)));
    CUDA_TRY(cudaMalloc(&c->ext_Ainv64, (size_t)2 * 36 * ge.Vh * sizeof(double2)));
    CUDA_TRY(cudaMalloc(&c->ext_A32, (size_t)2 * 18 * ge.Vh * sizeof(float4)));
    CUDA_TRY(cudaMalloc(&c->ext_Ainv32, (size_t)2 * 18 * ge.Vh * sizeof(float4)));
    CUDA_TRY(cudaMalloc(&c->ext_A16, (size_t)2 * 9 * ge.Vh * sizeof(uint4)));
    CUDA_TRY(cudaMalloc(&c->ext_Ainv16, (size_t)2 * 9 * ge.Vh * sizeof(uint4)));
    CUDA_TRY(cudaMalloc(&c->ext_logdet, (size_t)2 * 2 * ge.Vh * sizeof(double)));
  }
  {
    ProfScope ps(c, "clover_build", 0, 2.0 * ge.Vh * (60 * 216.0 + 2 * 1000.0));
    launch_pack_gauge(ge, c->U_ext, c->ext_g64, nullptr, 0, nullptr, 0, c->st);
    // every site of the extended lattice (the two outermost slices wrap and are discarded)
    launch_clover_build(ge, c->ext_g64, kappa, csw, c->ext_A64, c->ext_Ainv64, c->ext_A32, c->ext_Ainv32,
                        c->ext_A16, c->ext_Ainv16, work, c->ext_logdet, c->flags, c->st);
  }
  qcd_status s;
  if ((s = copy_slab_rows(c, c->A64, c->ext_A64, 36, sizeof(double2))) ||
      (s = copy_slab_rows(c, c->Ainv64, c->ext_Ainv64, 36, sizeof(double2))) ||
      (s = copy_slab_rows(c, c->A32, c->ext_A32, 18, sizeof(float4))) ||
      (s = copy_slab_rows(c, c->Ainv32, c->ext_Ainv32, 18, sizeof(float4))) ||
      (s = copy_slab_rows(c, c->A16, c->ext_A16, 9, sizeof(uint4))) ||
      (s = copy_slab_rows(c, c->Ainv16, c->ext_Ainv16, 9, sizeof(uint4))) ||
      (s = copy_slab_rows(c, c->logdet, c->ext_logdet, 2, sizeof(double))))
    return s;
  return QCD_OK;
}

qcd_status check_comm(const qcd_ctx* c, const qcd_slab_comm* m, int prec, int nrhs) {
  (void)c;
  (void)prec;
  (void)nrhs;
  if (!m || !m->send_lo || !m->send_hi || !m->recv_lo || !m->recv_hi || !m->exchange || !m->allreduce)
    return fail(QCD_ERR_ARG, "qcd_slab_comm needs four halo buffers, an exchange and an allreduce callback");
  return QCD_OK;
}

qcd_status comm_exchange(const qcd_slab_comm* m, size_t bytes) {
  if (m->exchange(m->user, bytes) != 0) return fail(QCD_ERR_COMM, "the halo exchange callback failed");
  return QCD_OK;
}

qcd_status comm_sum(const qcd_slab_comm* m, double* v, int n) {
  if (m->allreduce(m->user, v, n) != 0) return fail(QCD_ERR_COMM, "the allreduce callback failed");
  return QCD_OK;
}

// One hopping pass on the slab: pack the input's t-faces, exchange them, run the halo kernel.
qcd_status slab_pass(qcd_ctx* c, int prec, int epi, DslashArgs a, const qcd_slab_comm* m) {
  const int recon = recon_of(c, prec);
  launch_halo_pack(prec, recon, c->g, gauge_ptr(c, prec), a.in, a.in_norm, 1 - a.p, a.in_g5, m->send_lo, m->send_hi,
                   a.nrhs, c->st);
  qcd_status s = comm_exchange(m, halo_bytes(c, prec, a.nrhs));
  if (s) return s;
  a.halo_lo = m->recv_lo;
  a.halo_hi = m->recv_hi;
  double bytes, flops;
  dslash_cost(c, prec, epi, a.nrhs, &bytes, &flops);
  char name[40];
  snprintf(name, sizeof name, "dslash_slab_p%d_%s", prec,
           epi == EPI_NONE ? "plain" : (epi == EPI_CLOVER_INV ? "cloverinv" : "xpay"));
  ProfScope ps(c, name, bytes, flops);
  launch_dslash_halo(prec, recon, epi, a, c->st);
  return QCD_OK;
}

// out = Mhat in (dagger: Mhat^dag) on the slab's even sites; t: odd temporary; red: |out|^2 (FIN_STORE)
qcd_status slab_mhat(qcd_ctx* c, int prec, int nrhs, bool dagger, const void* in, const float* in_n, void* out,
                     float* out_n, void* t, float* t_n, const qcd_slab_comm* m, const ReduceArgs* red) {
  DslashArgs a = base_args(c, prec, 1, nrhs);
  a.in = in;
  a.in_norm = in_n;
  a.out = t;
  a.out_norm = t_n;
  a.clover = clover_ptr(c, prec, true, 1);
  a.in_g5 = dagger;
  qcd_status s = slab_pass(c, prec, EPI_CLOVER_INV, a, m);
  if (s) return s;
  DslashArgs b = base_args(c, prec, 0, nrhs);
  b.in = t;
  b.in_norm = t_n;
  b.out = out;
  b.out_norm = out_n;
  b.x = in;
  b.x_norm = in_n;
  b.clover = clover_ptr(c, prec, false, 0);
  b.a = -c->kappa * c->kappa;
  b.x_g5 = b.out_g5 = dagger;
  if (red) {
    b.do_norm = 1;
    b.red = *red;
  }
  return slab_pass(c, prec, EPI_XPAY, b, m);
}

qcd_status slab_mdagm(qcd_ctx* c, int prec, int nrhs, const void* in, const float* in_n, void* out, float* out_n,
                      void* t, float* t_n, void* y, float* y_n, const qcd_slab_comm* m, const ReduceArgs* red) {
  qcd_status s = slab_mhat(c, prec, nrhs, false, in, in_n, y, y_n, t, t_n, m, red);
  if (s) return s;
  return slab_mhat(c, prec, nrhs, true, y, y_n, out, out_n, t, t_n, m, nullptr);
}

// a reduction stored per RHS (FIN_STORE into c->results), summed over the slabs, then finalised in `mode`
qcd_status slab_finish(qcd_ctx* c, int mode, int nrhs, const qcd_slab_comm* m) {
  qcd_status s = comm_sum(m, c->results, nrhs);
  if (s) return s;
  launch_finalize(reduce_args(c, mode), c->results, nrhs, c->st);
  return QCD_OK;
}

// x_hi += x_lo, r = b - Mhat^dag Mhat x_hi in FP64 (the true residual, summed over the slabs), p = r + beta p
qcd_status slab_reliable(qcd_ctx* c, const SolverFields& f, int nrhs, const qcd_slab_comm* m) {
  const Geom& g = c->g;
  launch_accumulate_x(f.pr, g, nrhs, f.x_hi, f.x_lo, f.x_lo_n, c->st);
  qcd_status s = slab_mdagm(c, 64, nrhs, f.x_hi, nullptr, f.ap_hi, nullptr, f.t_hi, nullptr, f.y_hi, nullptr, m,
                            nullptr);
  if (s) return s;
  launch_true_residual(f.pr, g, nrhs, f.b_hi, f.ap_hi, f.r_lo, f.r_lo_n, reduce_args(c, FIN_STORE), c->st);
  if ((s = slab_finish(c, FIN_CG_TRUE, nrhs, m))) return s;
  launch_p_update(f.pr, f.pp, g, nrhs, f.r_lo, f.r_lo_n, f.p, f.p_n, c->cg, nullptr, c->st);
  return QCD_OK;
}

// The CG of cg_batch for one batch of slab fields, driven from the host: one look at the solver state
// per iteration (the exchanges and sums already return to the host between passes).
qcd_status slab_cg_batch(qcd_ctx* c, double2* x, const double2* b, int nrhs, const qcd_solver_params* prm,
                         qcd_solver_stats* stats, const qcd_slab_comm* m) {
  const Geom& g = c->g;
  SolverFields f;
  qcd_status s = solver_fields(c, prm->inner_prec, nrhs, &f);
  if (s) return s;
  const bool mixed = prm->inner_prec != 64;
  for (int r = 0; r < nrhs; r++) {
    CGState st;
    memset(&st, 0, sizeof st);
    st.tol2 = prm->tol * prm->tol;
    st.active = 1;
    st.reliable_updates = -1;
    c->h_cg[r] = st;
  }
  CGControl ctl;
  memset(&ctl, 0, sizeof ctl);
  ctl.reliable_every = mixed ? (prm->reliable_every > 0 ? prm->reliable_every : 50) : (1 << 30);
  ctl.delta2 = mixed ? prm->reliable_delta * prm->reliable_delta : 0.0;
  *c->h_ctl = ctl;
  CUDA_TRY(cudaMemcpyAsync(c->cg, c->h_cg, sizeof(CGState) * nrhs, cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(cudaMemcpyAsync(c->ctl, c->h_ctl, sizeof(CGControl), cudaMemcpyHostToDevice, c->st));
  launch_spinor_to_native(64, g, b, f.b_hi, nullptr, nrhs, c->st);
  launch_norm2(g, nrhs, f.b_hi, reduce_args(c, FIN_STORE), c->st);
  if ((s = slab_finish(c, FIN_CG_BNORM, nrhs, m))) return s;
  if (prm->use_x0) launch_spinor_to_native(64, g, x, f.x_hi, nullptr, nrhs, c->st);
  else launch_zero(f.x_hi, spinor_bytes(g, 64, nrhs), c->st);
  launch_zero(f.x_lo, spinor_bytes(g, f.pr, nrhs), c->st);
  launch_zero(f.p, spinor_bytes(g, f.pp, nrhs), c->st);
  if (f.p_n) launch_zero(f.p_n, sizeof(float) * (size_t)g.Vh * nrhs, c->st);
  // r = b - A x_hi (x_lo = 0, so the reliable update's accumulation adds nothing), p = r
  if ((s = slab_reliable(c, f, nrhs, m))) return s;
  qcd_status result = QCD_OK;
  bool stale = true;  // the host copy of the state predates the last reliable update
  while (true) {
    if (stale && (s = read_state(c, nrhs))) return s;
    if (c->h_ctl->overflow) return fail(QCD_ERR_CUDA, "reduction buffer too small (internal sizing error)");
    if (c->h_ctl->nan) {
      result = fail(QCD_ERR_NAN, "non-finite value or breakdown in CG");
      break;
    }
    bool active = false;
    int max_it = 0;
    for (int r = 0; r < nrhs; r++) {
      active |= c->h_cg[r].active != 0;
      max_it = std::max(max_it, c->h_cg[r].iters);
    }
    if (!active) break;
    if (max_it >= prm->max_iter) {
      result = fail(QCD_ERR_NOT_CONVERGED, "CG did not converge in %d iterations", prm->max_iter);
      if ((s = slab_reliable(c, f, nrhs, m))) return s;
      break;
    }
    // y = Mhat p, |y|^2 = <p, A p> -> alpha; Ap = Mhat^dag y; x += alpha p, r -= alpha Ap, |r|^2 -> beta
    ReduceArgs red = reduce_args(c, FIN_STORE);
    if ((s = slab_mhat(c, f.pp, nrhs, false, f.p, f.p_n, f.y, f.y_n, f.t, f.t_n, m, &red))) return s;
    if ((s = slab_finish(c, FIN_CG_PAP, nrhs, m))) return s;
    if ((s = slab_mhat(c, f.pp, nrhs, true, f.y, f.y_n, f.ap, f.ap_n, f.t, f.t_n, m, nullptr))) return s;
    launch_xr_update(f.pr, f.pp, g, nrhs, f.x_lo, f.r_lo, f.p, f.p_n, f.ap, f.ap_n, c->cg, reduce_args(c, FIN_STORE),
                     c->st);
    if ((s = slab_finish(c, FIN_CG_RR, nrhs, m))) return s;
    if ((s = read_state(c, nrhs))) return s;
    if (c->h_ctl->nan) {
      result = fail(QCD_ERR_NAN, "non-finite value or breakdown in CG");
      break;
    }
    if (c->h_ctl->halt) {
      // a reliable update (or the convergence check) is due for some RHS: it is made for all
      if ((s = slab_reliable(c, f, nrhs, m))) return s;
      stale = true;
    } else {
      // the p update leaves the state read above as it is
      launch_p_update(f.pr, f.pp, g, nrhs, f.r_lo, f.r_lo_n, f.p, f.p_n, c->cg, nullptr, c->st);
      stale = false;
    }
  }
  launch_accumulate_x(f.pr, g, nrhs, f.x_hi, f.x_lo, f.x_lo_n, c->st);
  launch_spinor_to_canon(64, g, f.x_hi, nullptr, x, nrhs, c->st);
  launch_redot(g, nrhs, f.b_hi, f.x_hi, reduce_args(c, FIN_STORE), c->st);
  if ((s = comm_sum(m, c->results, nrhs))) return s;
  CUDA_TRY(cudaMemcpyAsync(c->h_results, c->results, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->st));
  if ((s = read_state(c, nrhs))) return s;
  if (stats) {
    for (int r = 0; r < nrhs; r++) {
      const CGState& st = c->h_cg[r];
      stats[r].iters = st.iters;
      stats[r].reliable_updates = st.reliable_updates;
      stats[r].true_rel_resid = st.bnorm2 > 0 ? sqrt(st.true_rr / st.bnorm2) : 0.0;
      stats[r].b_dot_x = c->h_results[r];
    }
  }
  return result;
}

}  // namespace

extern "C" {

qcd_status qcd_create_slab(qcd_ctx** out, const int dims[4], int t_offset, int t_local, double t_bc,
                           void* stream) {
  nvtxRangePushA("qcd_create_slab");
  struct Pop {
    ~Pop() { nvtxRangePop(); }
  } pop;
  if (!out || !dims) return fail(QCD_ERR_ARG, "null argument");
  *out = nullptr;
  const int T = dims[3];
  if (T < 2 || T % 2) return fail(QCD_ERR_ARG, "extent 3 = %d must be even and >= 2", T);
  if (t_local < 2 || t_local % 2 || t_offset < 0 || t_offset % 2 || t_offset + t_local > T)
    return fail(QCD_ERR_ARG, "slab t_offset %d, t_local %d: both even, t_local >= 2, t_offset + t_local <= %d",
                t_offset, t_local, T);
  const int local[4] = {dims[0], dims[1], dims[2], t_local};
  qcd_ctx* c = nullptr;
  qcd_status s = create_ctx(&c, local, t_bc, stream);
  if (s) return s;
  c->slab = true;
  c->g.t0 = t_offset;
  c->g.Tg = T;
  c->ge = make_geom(dims[0], dims[1], dims[2], t_local + 4, t_bc, t_offset - 2, T);
  if ((long long)c->ge.Vh * 16 >= (1LL << 31)) {
    qcd_destroy(c);
    return fail(QCD_ERR_ARG, "slab too large");
  }
  *out = c;
  return QCD_OK;
}

qcd_status qcd_slab_halo_bytes(const qcd_ctx* c, int prec, int nrhs, size_t* bytes) {
  if (!c || !bytes) return fail(QCD_ERR_ARG, "null argument");
  if (!valid_prec(prec) || nrhs < 1) return fail(QCD_ERR_ARG, "precision 64/32/16 and nrhs >= 1");
  *bytes = halo_bytes(c, prec, std::min(nrhs, MAX_RHS));
  return QCD_OK;
}

qcd_status qcd_slab_dslash(qcd_ctx* c, double* out, const double* in, int op, int dagger, int prec, int nrhs,
                           const qcd_slab_comm* m) {
  QCD_API_ENTER("qcd_slab_dslash", c);
  qcd_status s = QCD_OK;
  if (!c->slab) return fail(QCD_ERR_STATE, "qcd_slab_dslash needs a context from qcd_create_slab");
  if (!out || !in) return fail(QCD_ERR_ARG, "null field pointer");
  if (op < QCD_OP_DSLASH_EO || op > QCD_OP_CLOVER_INV) return fail(QCD_ERR_ARG, "unknown op %d", op);
  if (!valid_prec(prec)) return fail(QCD_ERR_ARG, "precision must be 64, 32 or 16");
  if (nrhs < 1) return fail(QCD_ERR_ARG, "nrhs must be >= 1");
  if ((s = check_comm(c, m, prec, nrhs))) return s;
  if (!c->have_gauge) return fail(QCD_ERR_STATE, "dslash before load_gauge");
  if (op >= QCD_OP_MHAT && !c->have_clover) return fail(QCD_ERR_STATE, "op %d needs clover_build", op);
  const Geom& g = c->g;
  const size_t canon = (size_t)g.Vh * 12 * sizeof(double2);
  if ((const char*)out < (const char*)in + canon * nrhs && (const char*)in < (const char*)out + canon * nrhs)
    return fail(QCD_ERR_ARG, "in and out overlap");
  for (int done = 0; done < nrhs;) {
    const int nb = batch_of(nrhs - done);
    const double2* cin = reinterpret_cast<const double2*>(in) + (size_t)done * g.Vh * 12;
    double2* cout = reinterpret_cast<double2*>(out) + (size_t)done * g.Vh * 12;
    void *vin, *vout, *vt, *vy, *nin = nullptr, *nout = nullptr, *nt = nullptr, *ny = nullptr;
    const size_t fb = spinor_bytes(g, prec, nb), nbytes = sizeof(float) * (size_t)g.Vh * nb;
    if ((s = ws_get(c, S_IN, fb, &vin)) || (s = ws_get(c, S_OUT, fb, &vout)) || (s = ws_get(c, S_T, fb, &vt)) ||
        (s = ws_get(c, S_Y, fb, &vy)))
      return s;
    if (prec == 16) {
      if ((s = ws_get(c, S_IN_N, nbytes, &nin)) || (s = ws_get(c, S_OUT_N, nbytes, &nout)) ||
          (s = ws_get(c, S_T_N, nbytes, &nt)) || (s = ws_get(c, S_Y_N, nbytes, &ny)))
        return s;
    }
    float *fin = (float*)nin, *fout = (float*)nout, *ft = (float*)nt, *fy = (float*)ny;
    launch_spinor_to_native(prec, g, cin, vin, fin, nb, c->st);
    switch (op) {
      case QCD_OP_DSLASH_EO:
      case QCD_OP_DSLASH_OE: {
        DslashArgs a = base_args(c, prec, op == QCD_OP_DSLASH_EO ? 0 : 1, nb);
        a.in = vin;
        a.in_norm = fin;
        a.out = vout;
        a.out_norm = fout;
        a.in_g5 = a.out_g5 = dagger ? 1 : 0;
        s = slab_pass(c, prec, EPI_NONE, a, m);
        break;
      }
      case QCD_OP_MHAT:
        s = slab_mhat(c, prec, nb, dagger != 0, vin, fin, vout, fout, vt, ft, m, nullptr);
        break;
      case QCD_OP_MDAGM:
        s = slab_mdagm(c, prec, nb, vin, fin, vout, fout, vt, ft, vy, fy, m, nullptr);
        break;
      case QCD_OP_CLOVER:
        launch_clover_apply(prec, g, clover_ptr(c, prec, false, 0), vin, fin, vout, fout, nb, c->st);
        break;
      case QCD_OP_CLOVER_INV:
        launch_clover_apply(prec, g, clover_ptr(c, prec, true, 1), vin, fin, vout, fout, nb, c->st);
        break;
    }
    if (s) return s;
    launch_spinor_to_canon(prec, g, vout, fout, cout, nb, c->st);
    done += nb;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QCD_ERR_CUDA, "slab dslash launch: %s", cudaGetErrorString(e));
  return QCD_OK;
}

qcd_status qcd_slab_cg_solve(qcd_ctx* c, double* x, const double* b, int nrhs, const qcd_solver_params* prm,
                             qcd_solver_stats* stats, const qcd_slab_comm* m) {
  QCD_API_ENTER("qcd_slab_cg_solve", c);
  qcd_status s = QCD_OK;
  if (!c->slab) return fail(QCD_ERR_STATE, "qcd_slab_cg_solve needs a context from qcd_create_slab");
  if (!x || !b) return fail(QCD_ERR_ARG, "null field pointer");
  if (nrhs < 1) return fail(QCD_ERR_ARG, "nrhs must be >= 1");
  if ((s = check_params(prm))) return s;
  if ((s = check_comm(c, m, 64, nrhs))) return s;
  if (!c->have_clover) return fail(QCD_ERR_STATE, "cg_solve before clover_build");
  const auto t0 = std::chrono::steady_clock::now();
  const size_t fs = (size_t)c->g.Vh * 12;
  qcd_status worst = QCD_OK;
  for (int done = 0; done < nrhs;) {
    const int nb = batch_of(nrhs - done);
    s = slab_cg_batch(c, reinterpret_cast<double2*>(x) + done * fs, reinterpret_cast<const double2*>(b) + done * fs,
                      nb, prm, stats ? stats + done : nullptr, m);
    if (s == QCD_ERR_NOT_CONVERGED) worst = s;
    else if (s) return s;
    done += nb;
  }
  const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int r = 0; r < nrhs; r++) stats[r].seconds = sec;
  return worst;
}

}  // extern "C"
