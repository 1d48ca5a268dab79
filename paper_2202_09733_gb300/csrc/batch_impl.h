// Batched solver: many independent problems, one ESDIRK step for all of them.
// Included by lib.cu (it uses the context internals and the static helpers there).
//
// Problems with the same dimension, geometry degree and p-levels form a group, solved on
// one context whose mesh is the disjoint union of theirs (problem k of a group owns the
// element range [off_k, off_k + E_k)).  Every kernel of the step (residuals, Jv, element
// blocks, LU, pMG cycle, vector updates) then runs once per group instead of once per
// problem.  The Newton and FGMRES iterations stay per problem: norms and inner products
// are segmented reductions, each problem keeps its own Hessenberg matrix, Givens
// rotations, stopping test and restart, and a problem that has converged (or has not
// started) is masked out by zeroing its segment of the Krylov vectors, which every
// operator of the step maps to zero exactly.  So each problem goes through the same
// iteration as it would alone (the inner products differ from the one-problem reduction
// tree in rounding only).
//
// One Arnoldi step of a group (preconditioner, normalisation, Jv, two Gram-Schmidt
// passes, new basis vector) is one fixed sequence of kernels with no host round trip; it
// is captured once as a CUDA graph per (Krylov index, operator parameters) and replayed,
// and the host reads the step's scalars back once.

static const int kBatchLD = 64;     // per-problem stride of the device dot-product arrays
static const int kSegChunk = 2048;  // elements per reduction item

struct BGraph {
    cudaGraphExec_t exec;
    long long nkernels;
    // key
    int j, use_pmg, prec, nlev, ns[FRL_MAXLEV];
    double shift, eps, pmg_c;
    const double *q, *Rq;
};

struct BGroup {
    fr_ctx *C;
    int np;
    std::vector<int> probs, off, Ei;
    int *ep;                  // device: element -> problem index within the group
    int4 *items;
    int nitems;
    int *item_off;            // device [np + 1]
    double *partial;          // device [nitems][8]
    double *h1, *h2, *sq;     // device [np][kBatchLD] dot products; sq: scratch norms [np]
    double *nrm_z, *inv_z, *nrm_w, *inv_w, *nrm_x, *inv_x, *mask, *fac, *ydev;   // device [np] / [np][kBatchLD]
    double *Q;                // the group's working state
    double *target, *qref_dev;   // mixed cycle scaling held on the device
    std::vector<BGraph> graphs;
};

struct fr_batch {
    int nprob, d, nv;
    std::vector<BGroup> G;
    std::vector<int> group_of, index_in_group;
    int use_graphs;
    cudaStream_t st;
    cudaEvent_t ev;
};

static void batch_free_graphs(BGroup &g) {
    for (auto &x : g.graphs) cudaGraphExecDestroy(x.exec);
    g.graphs.clear();
}

extern "C" int fr_batch_destroy(fr_batch *B) {
    if (!B) return FR_OK;
    for (auto &g : B->G) {
        batch_free_graphs(g);
        fr_destroy(g.C);
    }
    if (B->ev) cudaEventDestroy(B->ev);
    if (B->st) cudaStreamDestroy(B->st);
    delete B;
    return FR_OK;
}

static bool same_structure(const fr_mesh_desc &a, const fr_mesh_desc &b) {
    if (a.dim != b.dim || a.qg != b.qg || a.nlevels != b.nlevels) return false;
    for (int l = 0; l < a.nlevels; ++l)
        if (a.plevels[l] != b.plevels[l]) return false;
    return true;
}

static int batch_build_group(fr_batch *B, BGroup &g, const fr_mesh_desc *meshes, const fr_physics *ph) {
    const fr_mesh_desc &m0 = meshes[g.probs[0]];
    int d = m0.dim, nn = (m0.qg + 1) * (m0.qg + 1) * (d == 3 ? m0.qg + 1 : 1);
    long long Et = 0, Ft = 0;
    for (int k : g.probs) { Et += meshes[k].nelem; Ft += meshes[k].nfaces; }
    if (Et > (1LL << 30) || Ft > (1LL << 30)) return fail(FR_ERR_INVALID_ARG, "batch group too large");
    std::vector<double> gn((size_t)Et * nn * d);
    std::vector<int> faces((size_t)Ft * 6);
    long long eo = 0, fo = 0;
    for (int k : g.probs) {
        const fr_mesh_desc &m = meshes[k];
        g.off.push_back((int)eo);
        g.Ei.push_back(m.nelem);
        memcpy(&gn[(size_t)eo * nn * d], m.gnodes, sizeof(double) * (size_t)m.nelem * nn * d);
        for (int f = 0; f < m.nfaces; ++f) {
            const int *src = m.faces + (size_t)f * 6;
            int *dst = &faces[(size_t)(fo + f) * 6];
            for (int c = 0; c < 6; ++c) dst[c] = src[c];
            if (src[0] < 0 || src[0] >= m.nelem || src[2] >= m.nelem)
                return fail(FR_ERR_INVALID_ARG, "problem %d: face %d names an element outside the mesh", k, f);
            dst[0] += (int)eo;
            if (src[2] >= 0) dst[2] += (int)eo;
        }
        eo += m.nelem;
        fo += m.nfaces;
    }
    fr_mesh_desc mg = m0;
    mg.nelem = (int)Et;
    mg.gnodes = gn.data();
    mg.nfaces = (int)Ft;
    mg.faces = faces.data();
    TRY(fr_create(&g.C, &mg, ph));
    fr_ctx *C = g.C;
    g.np = (int)g.probs.size();
    // element -> problem map and reduction items
    std::vector<int> ep((size_t)Et), ioff(g.np + 1);
    std::vector<int4> items;
    for (int k = 0; k < g.np; ++k) {
        for (int e = 0; e < g.Ei[k]; ++e) ep[(size_t)g.off[k] + e] = k;
        ioff[k] = (int)items.size();
        for (int e0 = 0; e0 < g.Ei[k]; e0 += kSegChunk)
            items.push_back(make_int4(k, g.off[k] + e0, g.off[k] + std::min(g.Ei[k], e0 + kSegChunk), 0));
    }
    ioff[g.np] = (int)items.size();
    g.nitems = (int)items.size();
    TRY(dalloc_t(C, &g.ep, (size_t)Et));
    TRY(dalloc_t(C, &g.items, items.size()));
    TRY(dalloc_t(C, &g.item_off, ioff.size()));
    CK(cudaMemcpy(g.ep, ep.data(), sizeof(int) * ep.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(g.items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(g.item_off, ioff.data(), sizeof(int) * ioff.size(), cudaMemcpyHostToDevice));
    TRY(dalloc_t(C, &g.partial, (size_t)g.nitems * 8));
    size_t pl = (size_t)g.np * kBatchLD;
    TRY(dalloc_t(C, &g.h1, pl)); TRY(dalloc_t(C, &g.h2, pl)); TRY(dalloc_t(C, &g.ydev, pl));
    TRY(dalloc_t(C, &g.sq, g.np));
    TRY(dalloc_t(C, &g.nrm_z, g.np)); TRY(dalloc_t(C, &g.inv_z, g.np));
    TRY(dalloc_t(C, &g.nrm_w, g.np)); TRY(dalloc_t(C, &g.inv_w, g.np));
    TRY(dalloc_t(C, &g.nrm_x, g.np)); TRY(dalloc_t(C, &g.inv_x, g.np));
    TRY(dalloc_t(C, &g.mask, g.np)); TRY(dalloc_t(C, &g.fac, g.np));
    TRY(dalloc_t(C, &g.Q, C->L[0].ndof));
    TRY(dalloc_t(C, &g.target, 1)); TRY(dalloc_t(C, &g.qref_dev, 5));
    return FR_OK;
}

extern "C" int fr_batch_create(fr_batch **out, int nprob, const fr_mesh_desc *meshes, const fr_physics *ph) {
    if (!out) return fail(FR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nprob < 1 || !meshes || !ph) return fail(FR_ERR_INVALID_ARG, "need at least one problem and physics");
    for (int k = 0; k < nprob; ++k) {
        const fr_mesh_desc &m = meshes[k];
        if ((m.dim != 2 && m.dim != 3) || m.nelem <= 0 || !m.gnodes || !m.faces || m.nfaces <= 0 || !m.plevels ||
            m.nlevels < 1 || m.nlevels > FRL_MAXLEV || (m.qg != 1 && m.qg != 2))
            return fail(FR_ERR_INVALID_ARG, "problem %d: invalid mesh description", k);
        if (m.dim != meshes[0].dim) return fail(FR_ERR_INVALID_ARG, "all problems of a batch share the dimension");
    }
    fr_batch *B = new fr_batch();
    B->nprob = nprob;
    B->d = meshes[0].dim;
    B->nv = B->d + 2;
    B->use_graphs = 1;
    B->group_of.assign(nprob, -1);
    B->index_in_group.assign(nprob, -1);
    for (int k = 0; k < nprob; ++k) {
        int gi = -1;
        for (size_t q = 0; q < B->G.size(); ++q)
            if (same_structure(meshes[B->G[q].probs[0]], meshes[k])) { gi = (int)q; break; }
        if (gi < 0) {
            B->G.emplace_back();
            gi = (int)B->G.size() - 1;
        }
        B->group_of[k] = gi;
        B->index_in_group[k] = (int)B->G[gi].probs.size();
        B->G[gi].probs.push_back(k);
    }
    for (auto &g : B->G) {
        int rc = batch_build_group(B, g, meshes, ph);
        if (rc != FR_OK) { fr_batch_destroy(B); return rc; }
    }
    if (cudaStreamCreateWithFlags(&B->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming) != cudaSuccess) {
        fr_batch_destroy(B);
        return fail(FR_ERR_CUDA, "creating the batch stream");
    }
    *out = B;
    return FR_OK;
}

extern "C" int fr_batch_info(const fr_batch *B, int *ngroups, int *group_of, int *elem_offset) {
    if (!B) return fail(FR_ERR_INVALID_ARG, "NULL batch");
    if (ngroups) *ngroups = (int)B->G.size();
    for (int k = 0; k < B->nprob; ++k) {
        if (group_of) group_of[k] = B->group_of[k];
        if (elem_offset) elem_offset[k] = B->G[B->group_of[k]].off[B->index_in_group[k]];
    }
    return FR_OK;
}

extern "C" int fr_batch_set_graphs(fr_batch *B, int on) {
    if (!B) return fail(FR_ERR_INVALID_ARG, "NULL batch");
    B->use_graphs = on ? 1 : 0;
    if (!on)
        for (auto &g : B->G) batch_free_graphs(g);
    return FR_OK;
}

// ------------------------------------------------------------ segmented helpers
static int seg_dots(BGroup &g, const double *w, int m, const double *const *V, double *out, int ld, cudaStream_t s) {
    const FrLevel &L = g.C->L[0];
    frkb_segdots(L.nd, L.E, g.nitems, g.items, g.np, g.item_off, w, m, V, g.partial, out, ld, s);
    CKLAUNCH();
    return FR_OK;
}
// per-problem norms of x into nrm (device) and mask/||x|| into inv (device)
static int seg_norm(BGroup &g, const double *x, const double *mask, double *nrm, double *inv, cudaStream_t s) {
    const double *V[1] = {x};
    TRY(seg_dots(g, x, 1, V, g.sq, 1, s));
    frkb_seg_invnorm(g.np, g.sq, 1, mask, nrm, inv, s);
    return FR_OK;
}
static void seg_scale(BGroup &g, const double *f, const double *x, double *y, cudaStream_t s) {
    frkb_seg_scale(g.C->L[0].ndof, g.C->L[0].E, g.ep, f, x, y, s);
}
static int to_host(double *h, const double *d, size_t n, cudaStream_t s) {
    CK(cudaMemcpyAsync(h, d, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    return FR_OK;
}

// preconditioner application without host round trips: the FP64 cycle as it is; the FP32
// cycle with its scale target kept on the device (one cycle per call, the gain measured by
// each call sets the next call's target)
static int pmg_apply_dev(fr_ctx *C, BGroup &g, const double *q, const double *Rq, const double *X, double *Y,
                         cudaStream_t s) {
    if (C->pmg_prec == 0) return pmg_apply(C, q, Rq, X, Y, s);
    long long n = C->L[0].ndof;
    PmgBuf<float> &P = C->p32;
    if (frk32_absmax(n, X, C->xmax, s) != 0) return fail(FR_ERR_CUDA, "absmax");
    frk32_d2f(n, q, C->q32, s);
    TRY(residual_t<float>(C, 0, C->q32, C->Rq32, s));
    frk32_d2f_scaled_dev(n, X, C->xmax, g.target, C->x32, s);
    frk32_copy(n, C->q32, P.qh[0], s);
    TRY(vcycle_t<float>(C, 0, C->q32, C->Rq32, C->x32, P.qh[0], s));
    frk32_sub(n, P.qh[0], C->q32, C->y32, s);
    frk32_f2d_unscale_dev(n, C->y32, C->xmax, g.target, Y, s);
    if (frk32_absmax_var_f(C->nv, n / C->nv, C->y32, C->ymax, s) != 0) return fail(FR_ERR_CUDA, "absmax");
    frk32_next_target(C->nv, C->ymax, g.qref_dev, kMixedAlpha, g.target, s);
    CKLAUNCH();
    return FR_OK;
}

// one Arnoldi step j for every problem of the group (device only; graph-capturable)
static int arnoldi_dev(BGroup &g, int j, const double *q, const double *Rq, const fr_gmres_opts *o, cudaStream_t s) {
    fr_ctx *C = g.C;
    long long n = C->L[0].ndof;
    const double *zj = C->V[j];
    if (o->use_pmg) {
        TRY(pmg_apply_dev(C, g, q, Rq, C->V[j], C->Z[j], s));
        TRY(seg_norm(g, C->Z[j], g.mask, g.nrm_z, g.inv_z, s));
        seg_scale(g, g.inv_z, C->Z[j], C->Z[j], s);
        zj = C->Z[j];
    }
    TRY(jvp(C, q, Rq, zj, o->eps, o->shift, C->gw, s));
    const double *const *Vp = (const double *const *)C->V.data();
    TRY(seg_dots(g, C->gw, j + 1, Vp, g.h1, kBatchLD, s));
    frkb_seg_multi_axpy(n, C->L[0].E, g.ep, j + 1, g.h1, kBatchLD, Vp, C->gw, s);
    TRY(seg_dots(g, C->gw, j + 1, Vp, g.h2, kBatchLD, s));
    frkb_seg_multi_axpy(n, C->L[0].E, g.ep, j + 1, g.h2, kBatchLD, Vp, C->gw, s);
    TRY(seg_norm(g, C->gw, g.mask, g.nrm_w, g.inv_w, s));
    seg_scale(g, g.inv_w, C->gw, C->V[j + 1], s);
    CKLAUNCH();
    return FR_OK;
}

static int arnoldi_step(fr_batch *B, BGroup &g, int j, const double *q, const double *Rq, const fr_gmres_opts *o,
                        cudaStream_t s) {
    if (!B->use_graphs) return arnoldi_dev(g, j, q, Rq, o, s);
    fr_ctx *C = g.C;
    for (auto &x : g.graphs) {
        bool same = x.j == j && x.use_pmg == o->use_pmg && x.shift == o->shift && x.eps == o->eps && x.q == q &&
                    x.Rq == Rq;
        if (same && o->use_pmg) {
            same = x.prec == C->pmg_prec && x.nlev == C->pmg_nlev && x.pmg_c == C->pmg_c;
            for (int l = 0; same && l < C->pmg_nlev; ++l) same = x.ns[l] == C->nsmooth[l];
        }
        if (same) {
            CK(cudaGraphLaunch(x.exec, s));
            g_graph_kernels += (unsigned long long)x.nkernels;
            return FR_OK;
        }
    }
    BGraph x;
    memset(&x, 0, sizeof x);
    x.j = j; x.use_pmg = o->use_pmg; x.shift = o->shift; x.eps = o->eps; x.q = q; x.Rq = Rq;
    x.prec = C->pmg_prec; x.nlev = C->pmg_nlev; x.pmg_c = C->pmg_c;
    for (int l = 0; l < FRL_MAXLEV; ++l) x.ns[l] = C->nsmooth[l];
    unsigned long long before = fr_kernel_launches();
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = arnoldi_dev(g, j, q, Rq, o, s);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc != FR_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return fail(FR_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    unsigned long long captured = fr_kernel_launches() - before;
    g_capture_kernels += captured;
    e = cudaGraphInstantiate(&x.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(FR_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    x.nkernels = (long long)captured;
    // one graph per Krylov index: a new key (another dt, level count, ...) replaces the old
    // graph of that index, so the cache stays at kdim graphs however often dt changes
    bool replaced = false;
    for (auto &y : g.graphs)
        if (y.j == j) {
            cudaGraphExecDestroy(y.exec);
            y = x;
            replaced = true;
            break;
        }
    if (!replaced) g.graphs.push_back(x);
    CK(cudaGraphLaunch(x.exec, s));
    g_graph_kernels += captured;
    return FR_OK;
}

// per-problem FGMRES(K), right-preconditioned, CGS2, in lockstep over the group's problems.
// active[k] = 0 leaves problem k out (its x stays 0).  b, x: group vectors.
struct BStats { std::vector<int> iters, restarts; std::vector<double> relres; };

static int gmres_batched(fr_batch *B, BGroup &g, const double *q, const double *Rq, const double *b, double *x,
                         const fr_gmres_opts *o, const std::vector<int> &want, BStats &bs, cudaStream_t s) {
    fr_ctx *C = g.C;
    int K = o->kdim, np = g.np;
    TRY(gmres_alloc(C, K));
    long long n = C->L[0].ndof;
    double *r = C->gr;
    std::vector<double> H((size_t)np * (K + 1) * K), cs((size_t)np * K), sn((size_t)np * K), gv((size_t)np * (K + 1));
    std::vector<double> bnorm(np), beta(np), est(np), mask(np), h1((size_t)np * kBatchLD), h2((size_t)np * kBatchLD),
        nw(np), nz(np), y((size_t)np * kBatchLD);
    std::vector<int> done(np), act(np), jj(np), total(np, 0), rest(np, 0);
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    for (int k = 0; k < np; ++k) mask[k] = want[k] ? 1.0 : 0.0;
    CK(cudaMemcpyAsync(g.mask, mask.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
    TRY(seg_norm(g, b, g.mask, g.nrm_x, g.inv_x, s));
    TRY(to_host(bnorm.data(), g.nrm_x, np, s));
    CK(cudaStreamSynchronize(s));
    for (int k = 0; k < np; ++k) {
        if (!want[k]) bnorm[k] = 0.0;
        if (!isfinite(bnorm[k])) return fail(FR_ERR_NONFINITE, "non-finite right-hand side (problem %d)", g.probs[k]);
        beta[k] = est[k] = bnorm[k];
        done[k] = bnorm[k] == 0.0;
    }
    // V0 = b / ||b|| per problem (inv_x holds mask / ||b||)
    seg_scale(g, g.inv_x, b, C->V[0], s);
    std::vector<const double *> Zp(K);
    for (;;) {
        int any = 0;
        for (int k = 0; k < np; ++k) {
            act[k] = !done[k];
            any |= act[k];
            jj[k] = 0;
            for (int i = 0; i <= K; ++i) gv[(size_t)k * (K + 1) + i] = 0.0;
            gv[(size_t)k * (K + 1)] = beta[k];
        }
        if (!any) break;
        for (int j = 0; j < K; ++j) {
            for (int k = 0; k < np; ++k) mask[k] = act[k] ? 1.0 : 0.0;
            CK(cudaMemcpyAsync(g.mask, mask.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
            TRY(arnoldi_step(B, g, j, q, Rq, o, s));
            Zp[j] = o->use_pmg ? C->Z[j] : C->V[j];
            TRY(to_host(h1.data(), g.h1, (size_t)np * kBatchLD, s));
            TRY(to_host(h2.data(), g.h2, (size_t)np * kBatchLD, s));
            TRY(to_host(nw.data(), g.nrm_w, np, s));
            if (o->use_pmg) TRY(to_host(nz.data(), g.nrm_z, np, s));
            CK(cudaStreamSynchronize(s));
            int still = 0;
            for (int k = 0; k < np; ++k) {
                if (!act[k]) continue;
                if (o->use_pmg && (!(nz[k] > 0.0) || !isfinite(nz[k])))
                    return fail(FR_ERR_NONFINITE, "preconditioner output norm %g (problem %d)", nz[k], g.probs[k]);
                if (!isfinite(nw[k])) return fail(FR_ERR_NONFINITE, "non-finite Arnoldi vector (problem %d)", g.probs[k]);
                double *Hk = &H[(size_t)k * (K + 1) * K], *ck = &cs[(size_t)k * K], *sk = &sn[(size_t)k * K];
                double *gk = &gv[(size_t)k * (K + 1)];
                for (int i = 0; i <= j; ++i) Hk[(size_t)i * K + j] = h1[(size_t)k * kBatchLD + i] + h2[(size_t)k * kBatchLD + i];
                double hn = nw[k];
                Hk[(size_t)(j + 1) * K + j] = hn;
                for (int i = 0; i < j; ++i) {
                    double a = Hk[(size_t)i * K + j], bb = Hk[(size_t)(i + 1) * K + j];
                    Hk[(size_t)i * K + j] = ck[i] * a + sk[i] * bb;
                    Hk[(size_t)(i + 1) * K + j] = -sk[i] * a + ck[i] * bb;
                }
                double a = Hk[(size_t)j * K + j], bb = Hk[(size_t)(j + 1) * K + j];
                double rr = hypot(a, bb);
                ck[j] = a / rr; sk[j] = bb / rr;
                Hk[(size_t)j * K + j] = rr; Hk[(size_t)(j + 1) * K + j] = 0.0;
                gk[j + 1] = -sk[j] * gk[j];
                gk[j] = ck[j] * gk[j];
                ++total[k];
                jj[k] = j + 1;
                est[k] = fabs(gk[j + 1]);
                if (est[k] <= o->tol * bnorm[k] || total[k] >= o->maxit || hn == 0.0) act[k] = 0;
                still |= act[k];
            }
            if (!still) break;
        }
        // x += Z y per problem
        int mmax = 0;
        for (int k = 0; k < np; ++k) {
            double *yk = &y[(size_t)k * kBatchLD];
            for (int i = 0; i < kBatchLD; ++i) yk[i] = 0.0;
            if (done[k] || jj[k] == 0) continue;
            const double *Hk = &H[(size_t)k * (K + 1) * K], *gk = &gv[(size_t)k * (K + 1)];
            for (int i = jj[k] - 1; i >= 0; --i) {
                double sacc = gk[i];
                for (int c = i + 1; c < jj[k]; ++c) sacc -= Hk[(size_t)i * K + c] * yk[c];
                yk[i] = sacc / Hk[(size_t)i * K + i];
            }
            mmax = std::max(mmax, jj[k]);
        }
        if (mmax > 0) {
            CK(cudaMemcpyAsync(g.ydev, y.data(), sizeof(double) * y.size(), cudaMemcpyHostToDevice, s));
            frkb_seg_update_x(n, C->L[0].E, g.ep, mmax, g.ydev, kBatchLD, Zp.data(), x, s);
            CKLAUNCH();
        }
        int again = 0;
        for (int k = 0; k < np; ++k) {
            if (done[k]) continue;
            if (est[k] <= o->tol * bnorm[k] || total[k] >= o->maxit) done[k] = 1;
            else again = 1;
        }
        if (!again) break;
        // restart: true residual b - A x of the problems still running
        for (int k = 0; k < np; ++k) mask[k] = done[k] ? 0.0 : 1.0;
        CK(cudaMemcpyAsync(g.mask, mask.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
        TRY(seg_norm(g, x, g.mask, g.nrm_x, g.inv_x, s));
        seg_scale(g, g.inv_x, x, r, s);
        TRY(jvp(C, q, Rq, r, o->eps, o->shift, C->gw, s));
        seg_scale(g, g.nrm_x, C->gw, C->gtmp, s);
        frk64_sub(n, b, C->gtmp, r, s);
        TRY(seg_norm(g, r, g.mask, g.nrm_w, g.inv_w, s));
        TRY(to_host(beta.data(), g.nrm_w, np, s));
        CK(cudaStreamSynchronize(s));
        for (int k = 0; k < np; ++k) {
            if (done[k]) continue;
            if (!isfinite(beta[k])) return fail(FR_ERR_NONFINITE, "non-finite GMRES residual (problem %d)", g.probs[k]);
            ++rest[k];
        }
        seg_scale(g, g.inv_w, r, C->V[0], s);
    }
    CK(cudaStreamSynchronize(s));
    for (int k = 0; k < np; ++k) {
        bs.iters[k] += total[k];
        bs.restarts[k] += rest[k];
        bs.relres[k] = bnorm[k] > 0.0 ? est[k] / bnorm[k] : 0.0;
    }
    return FR_OK;
}

// one ESDIRK step of every problem of group g on its working state g.Q
static int esdirk_group(fr_batch *B, BGroup &g, const fr_esdirk_tableau *tab, double dt, const fr_solve_opts *o,
                        fr_step_stats *stats, cudaStream_t s) {
    fr_ctx *C = g.C;
    int ns = tab->stages, np = g.np;
    TRY(stepper_alloc(C, ns + 5));
    long long n = C->L[0].ndof;
    double *q = g.Q, *qn = C->stv[0], *sv = C->stv[1], *F = C->stv[2], *Rk = C->stv[3], *dq = C->stv[4];
    double **Rs = &C->stv[5];
    std::vector<double> ndof(np), res(np), fs(np), fac(np);
    for (int k = 0; k < np; ++k) ndof[k] = (double)C->L[0].nd * g.Ei[k];
    std::vector<int> nptc(np, 0), conv_all(np, 1), conv(np);
    BStats bs;
    bs.iters.assign(np, 0); bs.restarts.assign(np, 0); bs.relres.assign(np, 0.0);
    frk64_copy(n, q, qn, s);
    TRY(residual(C, 0, qn, Rs[0], s));
    double aii = tab->A[1 * ns + 1];
    double c = 1.0 / o->dtau + 1.0 / (aii * dt);
    if (o->use_pmg) {
        fr_pmg_opts po;
        po.nlevels = o->nlevels;
        for (int l = 0; l < 4; ++l) po.nsmooth[l] = o->nsmooth[l];
        po.c = c;
        po.inv_dtau_star = o->inv_dtau_star;
        po.precision = o->precision;
        coarse_opts_copy(o, &po);
        TRY(pmg_setup_(C, qn, &po, s));
        if (o->precision == 1) {
            // device-held scale of the FP32 cycle: its first target from the setup's gain
            double t0 = kMixedAlpha / C->pmg_gain;
            CK(cudaMemcpyAsync(g.target, &t0, sizeof(double), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(g.qref_dev, C->pmg_qref, sizeof(double) * C->nv, cudaMemcpyHostToDevice, s));
            CK(cudaStreamSynchronize(s));
        }
    }
    fr_gmres_opts go = gm_opts(o, c);
    std::vector<int> want(np);
    for (int i = 1; i < ns; ++i) {
        double adt = tab->A[i * ns + i] * dt;
        double coef[6];
        for (int j = 0; j < i; ++j) coef[j] = tab->A[i * ns + j];
        frk64_lincomb(n, i, coef, (const double *const *)Rs, qn, dt, sv, s);
        frk64_copy(n, qn, q, s);
        for (int k = 0; k < np; ++k) conv[k] = 0;
        for (int it = 0; it <= o->max_ptc; ++it) {
            TRY(residual(C, 0, q, Rk, s));
            frk64_stage_F(n, q, sv, adt, Rk, F, s);
            const double *V1[1] = {F};
            TRY(seg_dots(g, F, 1, V1, g.sq, 1, s));
            TRY(to_host(fs.data(), g.sq, np, s));
            CK(cudaStreamSynchronize(s));
            int left = 0;
            for (int k = 0; k < np; ++k) {
                res[k] = fabs(adt) * sqrt(fs[k]) / sqrt(ndof[k]);
                if (!isfinite(res[k]))
                    return fail(FR_ERR_NONFINITE, "non-finite stage residual (problem %d, stage %d)", g.probs[k], i);
                if (!conv[k] && res[k] <= o->tol_newton) conv[k] = 1;
                left |= !conv[k];
            }
            if (!left || it == o->max_ptc) break;
            // -F on the problems still iterating, 0 on the converged ones
            for (int k = 0; k < np; ++k) { fac[k] = conv[k] ? 0.0 : -1.0; want[k] = !conv[k]; }
            CK(cudaMemcpyAsync(g.fac, fac.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
            seg_scale(g, g.fac, F, F, s);
            TRY(gmres_batched(B, g, q, Rk, F, dq, &go, want, bs, s));
            frk64_add(n, q, dq, q, s);
            for (int k = 0; k < np; ++k) nptc[k] += !conv[k];
        }
        for (int k = 0; k < np; ++k) {
            if (!conv[k]) conv_all[k] = 0;
            stats[k].final_res = res[k];
        }
        frk64_copy(n, Rk, Rs[i], s);
    }
    frk64_lincomb(n, ns, tab->b, (const double *const *)Rs, qn, dt, q, s);
    CKLAUNCH();
    for (int k = 0; k < np; ++k) {
        stats[k].n_ptc = nptc[k];
        stats[k].n_gmres = bs.iters[k];
        stats[k].converged = conv_all[k];
    }
    return FR_OK;
}

extern "C" int fr_batch_esdirk_step(fr_batch *B, const fr_esdirk_tableau *tab, double dt, double *const *q,
                                    const fr_solve_opts *o, fr_step_stats *stats, void *stream) {
    if (!B || !tab || !q || !o) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    if (tab->stages < 2 || tab->stages > 6 || !(dt > 0.0)) return fail(FR_ERR_INVALID_ARG, "bad tableau or dt");
    if (o->guess != 0 || o->train_iters != 0)
        return fail(FR_ERR_UNIMPLEMENTED, "the batched step starts every stage from q^n (guess 0, no training)");
    if (o->nonlinear != 0)
        return fail(FR_ERR_UNIMPLEMENTED, "the batched step solves its stages by JFNK (nonlinear 0)");
    if (o->use_pmg && o->coarse_smoother != 0)
        return fail(FR_ERR_UNIMPLEMENTED, "the matrix-based coarse smoother's inner products would couple the problems "
                                          "of a group; batched steps smooth with element-Jacobi blocks");
    if (o->kdim > kBatchLD - 2) return fail(FR_ERR_INVALID_ARG, "batched FGMRES needs kdim <= %d", kBatchLD - 2);
    for (int k = 0; k < B->nprob; ++k)
        if (!q[k]) return fail(FR_ERR_INVALID_ARG, "state of problem %d is NULL", k);
    // each group takes at most as many pMG levels as it has
    std::vector<fr_solve_opts> og(B->G.size(), *o);
    for (size_t gi = 0; gi < B->G.size(); ++gi) {
        og[gi].nlevels = std::min(o->nlevels, B->G[gi].C->nlev);
        TRY(check_solve_opts(B->G[gi].C, &og[gi]));
    }
    cudaStream_t us = S_(stream), s = B->st;
    CK(cudaEventRecord(B->ev, us));
    CK(cudaStreamWaitEvent(s, B->ev, 0));
    std::vector<fr_step_stats> loc(B->nprob);
    memset(loc.data(), 0, sizeof(fr_step_stats) * loc.size());
    for (size_t gi = 0; gi < B->G.size(); ++gi) {
        BGroup &g = B->G[gi];
        const FrLevel &L = g.C->L[0];
        for (int k = 0; k < g.np; ++k) frkb_gather(L.nd, g.Ei[k], q[g.probs[k]], g.Q, L.E, g.off[k], s);
        std::vector<fr_step_stats> gs(g.np);
        memset(gs.data(), 0, sizeof(fr_step_stats) * gs.size());
        TRY(esdirk_group(B, g, tab, dt, &og[gi], gs.data(), s));
        for (int k = 0; k < g.np; ++k) {
            frkb_scatter(L.nd, g.Ei[k], g.Q, L.E, g.off[k], q[g.probs[k]], s);
            loc[g.probs[k]] = gs[k];
            loc[g.probs[k]].prec_switch_it = -1;
        }
        CKLAUNCH();
    }
    CK(cudaEventRecord(B->ev, s));
    CK(cudaStreamWaitEvent(us, B->ev, 0));
    CK(cudaStreamSynchronize(s));
    int allc = 1;
    for (int k = 0; k < B->nprob; ++k) allc &= loc[k].converged;
    if (stats) memcpy(stats, loc.data(), sizeof(fr_step_stats) * loc.size());
    return allc ? FR_OK : fail(FR_ERR_NOT_CONVERGED, "a problem did not reach the Newton tolerance");
}

// R(q_k) of every problem (one residual per group); q, R: host arrays of device pointers
extern "C" int fr_batch_residual(fr_batch *B, double *const *q, double *const *R, void *stream) {
    if (!B || !q || !R) return fail(FR_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t us = S_(stream), s = B->st;
    CK(cudaEventRecord(B->ev, us));
    CK(cudaStreamWaitEvent(s, B->ev, 0));
    for (auto &g : B->G) {
        fr_ctx *C = g.C;
        TRY(stepper_alloc(C, 1));
        const FrLevel &L = C->L[0];
        for (int k = 0; k < g.np; ++k) {
            if (!q[g.probs[k]] || !R[g.probs[k]]) return fail(FR_ERR_INVALID_ARG, "NULL state");
            frkb_gather(L.nd, g.Ei[k], q[g.probs[k]], g.Q, L.E, g.off[k], s);
        }
        TRY(residual(C, 0, g.Q, C->stv[0], s));
        for (int k = 0; k < g.np; ++k) frkb_scatter(L.nd, g.Ei[k], C->stv[0], L.E, g.off[k], R[g.probs[k]], s);
        CKLAUNCH();
    }
    CK(cudaEventRecord(B->ev, s));
    CK(cudaStreamWaitEvent(us, B->ev, 0));
    return FR_OK;
}

extern "C" int fr_batch_autotune(fr_batch *B, int flags, int reps, char *report, int report_len) {
    if (!B) return fail(FR_ERR_INVALID_ARG, "NULL batch");
    if (report && report_len > 0) report[0] = 0;
    for (auto &g : B->G) {
        size_t u = report ? strlen(report) : 0;
        TRY(fr_autotune(g.C, flags, reps, report ? report + u : nullptr, report ? report_len - (int)u : 0));
        batch_free_graphs(g);   // captured graphs hold the old launch shapes
    }
    return FR_OK;
}
