// C ABI of libam (declared in include/am.h): argument checks, device memory,
// set-up precomputation and the call sequence of a solve and of a step.
#include "am_internal.cuh"
#include "ops.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

namespace am {
const char* thread_error();
}

namespace {

int set_err(am_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return set_err(h, AM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}
cudaError_t balloc(void** p, size_t bytes) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    return cudaMalloc(p, std::max<size_t>(bytes, 16));
}
template <class T>
void dfree(T** p) {
    if (*p) cudaFree(*p);
    *p = nullptr;
}
template <class T>
cudaError_t h2d(T* d, const T* hsrc, size_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    return cudaMemcpyAsync(d, hsrc, count * sizeof(T), cudaMemcpyHostToDevice, s);
}
template <class T>
cudaError_t d2h(T* hdst, const T* d, size_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    return cudaMemcpyAsync(hdst, d, count * sizeof(T), cudaMemcpyDeviceToHost, s);
}

// Host rotation R(theta) v (App. B, Eq. rot_mat), for set-up only.
void host_rotate(const double* th, const double* v, double* o, bool transpose) {
    const double s = th[0];
    const double sg = transpose ? -1.0 : 1.0;
    const double p[3] = {sg * th[1], sg * th[2], sg * th[3]};
    const double pv = p[0] * v[0] + p[1] * v[1] + p[2] * v[2];
    const double c[3] = {p[1] * v[2] - p[2] * v[1], p[2] * v[0] - p[0] * v[2], p[0] * v[1] - p[1] * v[0]};
    const double k = s * s - 0.5;
    for (int a = 0; a < 3; ++a) o[a] = 2.0 * (p[a] * pv + s * c[a] + k * v[a]);
}

// Inverse of a small dense n x n matrix by Gauss-Jordan with partial
// pivoting; false if singular.
bool host_inverse(std::vector<double>& A, int n) {
    std::vector<double> I(static_cast<size_t>(n) * n, 0.0);
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
        if (!(std::fabs(A[(size_t)piv * n + c]) > 1e-300)) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(A[(size_t)piv * n + k], A[(size_t)c * n + k]);
                std::swap(I[(size_t)piv * n + k], I[(size_t)c * n + k]);
            }
        const double d = 1.0 / A[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) { A[(size_t)c * n + k] *= d; I[(size_t)c * n + k] *= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
                I[(size_t)r * n + k] -= f * I[(size_t)c * n + k];
            }
        }
    }
    A.swap(I);
    return true;
}

// Order of the per-body or per-articulated-body preconditioner builds:
// matrices of at most two 32-row tiles (rows[i] <= 64) first, one CTA each,
// then the larger ones, built by clusters of cs CTAs: cs doubles (up to 8)
// while the larger ones' clusters still fit twice the SM count.
void split_for_build(const std::vector<int>& rows, std::vector<int>& list, int& n_small, int& cs) {
    const int n = (int)rows.size();
    list.clear();
    for (int i = 0; i < n; ++i)
        if (rows[i] <= 2 * 32) list.push_back(i);
    n_small = (int)list.size();
    for (int i = 0; i < n; ++i)
        if (rows[i] > 2 * 32) list.push_back(i);
    const long long large = n - n_small;
    cs = 1;
    while (cs < 8 && large > 0 && large * cs * 2 <= 2LL * am::num_sms()) cs *= 2;
}

void free_links(am_handle* h) {
    dfree(&h->d_bp); dfree(&h->d_bq); dfree(&h->d_dlp); dfree(&h->d_dlq);
    dfree(&h->d_dlpd); dfree(&h->d_dlqd); dfree(&h->d_dlp1); dfree(&h->d_dlq1);
    dfree(&h->d_lp); dfree(&h->d_lq); dfree(&h->d_B);
    dfree(&h->d_body_link_off); dfree(&h->d_body_link_idx);
    dfree(&h->d_asm_link_off); dfree(&h->d_asm_link_idx); dfree(&h->d_link_local);
    dfree(&h->d_pplus); dfree(&h->d_pplus_off);
    dfree(&h->d_G); dfree(&h->d_Gwork); dfree(&h->d_G_off); dfree(&h->d_G_rank);
    dfree(&h->d_perm); dfree(&h->d_perm_off);
    dfree(&h->d_corr); dfree(&h->d_corr_off); dfree(&h->d_zbuf); dfree(&h->d_cbuf);
    dfree(&h->d_pca_asm); dfree(&h->d_pca_chunk); dfree(&h->d_pca_list);
    h->n_pca = 0;
    h->n_pca_small = 0;
    h->pca_cs = 1;
}

void free_bodies(am_handle* h) {
    dfree(&h->d_q); dfree(&h->d_theta); dfree(&h->d_rho); dfree(&h->d_F); dfree(&h->d_slip);
    dfree(&h->d_blob_off); dfree(&h->d_body_of_blob); dfree(&h->d_asm_of_body);
    dfree(&h->d_asm_body_off); dfree(&h->d_asm_body_idx); dfree(&h->d_body_local);
    dfree(&h->d_r4); dfree(&h->d_d4); dfree(&h->d_rhi); dfree(&h->d_rlo); dfree(&h->d_r3);
    dfree(&h->d_minv); dfree(&h->d_pcwork); dfree(&h->d_Y); dfree(&h->d_Nt); dfree(&h->d_minv_off);
    dfree(&h->d_pc_w); dfree(&h->d_pc_Uhat); dfree(&h->d_mv);
    dfree(&h->d_pcw_body); dfree(&h->d_pcw_chunk); dfree(&h->d_pcw_off); dfree(&h->d_ytp); dfree(&h->d_pcb_cnt);
    dfree(&h->d_pcb_list);
    h->n_pcb_small = 0;
    h->pcb_cs = 1;
    h->n_pcw = 0;
    dfree(&h->d_qnew); dfree(&h->d_thnew); dfree(&h->d_iters); dfree(&h->d_q0); dfree(&h->d_th0); dfree(&h->d_fst); dfree(&h->d_sbpart);
}

void free_solver(am_handle* h) {
    dfree(&h->d_b); dfree(&h->d_x); dfree(&h->d_xhist); dfree(&h->d_t); dfree(&h->d_z);
    dfree(&h->d_w); dfree(&h->d_V); dfree(&h->d_Z); dfree(&h->d_rir); dfree(&h->d_dx);
    dfree(&h->d_vj); dfree(&h->d_zj);
    h->layout_gen++;
    dfree(&h->d_Hm); dfree(&h->d_cs); dfree(&h->d_sn); dfree(&h->d_g); dfree(&h->d_coef);
    dfree(&h->d_xi); dfree(&h->d_part); dfree(&h->d_npart);
    dfree(&h->d_sys_of_elem); dfree(&h->d_sys_of_blob); dfree(&h->d_sys_body_off); dfree(&h->d_chunk_start); dfree(&h->d_chunk_end);
    dfree(&h->d_sys_chunk_off); dfree(&h->d_Hs); dfree(&h->d_css); dfree(&h->d_sns); dfree(&h->d_gs);
    dfree(&h->d_coefs); dfree(&h->d_xis); dfree(&h->d_hcols); dfree(&h->d_bnorm_s); dfree(&h->d_beta_s);
    dfree(&h->d_inv_s); dfree(&h->d_tol_s); dfree(&h->d_sysred); dfree(&h->d_active); dfree(&h->d_kdone);
    dfree(&h->d_sys_blob0); dfree(&h->d_sys_nb); dfree(&h->d_sys_nch); dfree(&h->d_sys_poff);
    dfree(&h->d_item_counter); dfree(&h->d_arn_cnt);
    if (h->d_items) cudaFree(h->d_items);
    h->d_items = nullptr;
    h->n_items = 0;
    if (h->d_sym_items) cudaFree(h->d_sym_items);
    h->d_sym_items = nullptr;
    h->n_sym = 0;
}

int alloc_solver(am_handle* h) {
    const int n = h->n;
    const int m = h->restart;
    h->ldv = (n + 31) & ~31;
    CK(dalloc(&h->d_b, n)); CK(dalloc(&h->d_x, n)); CK(dalloc(&h->d_xhist, 3 * (size_t)n));
    CK(dalloc(&h->d_t, n)); CK(dalloc(&h->d_z, n)); CK(dalloc(&h->d_w, n));
    CK(dalloc(&h->d_rir, n)); CK(dalloc(&h->d_dx, n));
    CK(dalloc(&h->d_V, (size_t)h->ldv * (m + 1)));
    CK(dalloc(&h->d_vj, n)); CK(dalloc(&h->d_zj, n));
    h->layout_gen++;
    CK(dalloc(&h->d_Z, (size_t)h->ldv * m));
    CK(dalloc(&h->d_Hm, (size_t)(m + 1) * m)); CK(dalloc(&h->d_cs, m)); CK(dalloc(&h->d_sn, m));
    CK(dalloc(&h->d_g, m + 1)); CK(dalloc(&h->d_coef, m + 1)); CK(dalloc(&h->d_xi, m + 1));
    CK(dalloc(&h->d_part, (size_t)(m + 1) * 64)); CK(dalloc(&h->d_npart, 4 * am::num_sms() + 64));
    h->n_hist = 0;
    h->hist_head = 0;
    return AM_OK;
}

// Weights w[0..k) of the Lagrange polynomial through the nodes tn[0..k),
// evaluated at t.
void lagrange_weights(const double* tn, int k, double t, double* w) {
    for (int i = 0; i < k; ++i) {
        double v = 1.0;
        for (int j = 0; j < k; ++j)
            if (j != i) v *= (t - tn[j]) / (tn[i] - tn[j]);
        w[i] = v;
    }
}

// The initial guess of a time-step solve at time t from the history into x
// (am_set_initial_guess); false if the history is not used.
bool guess_from_history(am_handle* h, double t, double* x) {
    if (h->guess_order < 1 || h->n_hist < 1) return false;
    const double* slot[3];
    double tn[3];
    for (int i = 0; i < h->n_hist; ++i) {
        const int k = (h->hist_head - i + 3) % 3;
        slot[i] = h->d_xhist + (size_t)k * h->n;
        tn[i] = h->t_hist[k];
    }
    int k = std::min(h->guess_order, h->n_hist);
    double w[3] = {1.0, 0.0, 0.0};
    for (; k > 1; --k) {
        bool ok = true;
        const double sep = 1e-12 * (1.0 + std::fabs(t));
        for (int i = 0; i < k && ok; ++i)
            for (int j = i + 1; j < k && ok; ++j) ok = std::fabs(tn[i] - tn[j]) > sep;
        if (!ok) continue;
        lagrange_weights(tn, k, t, w);
        for (int i = 0; i < k; ++i) ok = ok && std::isfinite(w[i]) && std::fabs(w[i]) <= 16.0;
        if (ok) break;
    }
    if (k <= 1) {
        cudaMemcpyAsync(x, slot[0], h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    } else {
        // lambda and U extrapolated; phi from the newest solution (with a
        // rank-deficient C each solve's phi is one representative modulo
        // null(C^T), and those of different solves need not lie on one
        // smooth curve)
        const int n_phi = 3 * h->P;
        am::combine_vectors(h, x, slot, w, k, h->n - n_phi);
        cudaMemcpyAsync(x + (h->n - n_phi), slot[0] + (h->n - n_phi), n_phi * sizeof(double),
                        cudaMemcpyDeviceToDevice, h->stream);
    }
    return true;
}

// Append the solution of a time-step solve at time t to the history (a
// solve at the time of the most recent entry replaces it).
void push_history(am_handle* h, double t, const double* x) {
    if (!(h->n_hist > 0 && h->t_hist[h->hist_head] == t)) {
        h->hist_head = (h->hist_head + 1) % 3;
        h->n_hist = std::min(h->n_hist + 1, 3);
    }
    h->t_hist[h->hist_head] = t;
    cudaMemcpyAsync(h->d_xhist + (size_t)h->hist_head * h->n, x, h->n * sizeof(double),
                    cudaMemcpyDeviceToDevice, h->stream);
}

// Links and everything that depends on them.  Empty (P = 0) is valid.
int build_links(am_handle* h, int P, const int* bp, const int* bq) {
    const int M = h->M, NA = h->NA;
    free_links(h);
    h->layout_gen++;
    h->P = P;
    h->bp.assign(bp, bp + P);
    h->bq.assign(bq, bq + P);
    // body -> link CSR (code = 2 n + side, side 1 = the link's body q)
    std::vector<int> bl_off(M + 1, 0), bl_idx(2 * (size_t)P);
    for (int n = 0; n < P; ++n) { bl_off[bp[n] + 1]++; bl_off[bq[n] + 1]++; }
    for (int p = 0; p < M; ++p) bl_off[p + 1] += bl_off[p];
    {
        std::vector<int> fill(bl_off.begin(), bl_off.end() - 1);
        for (int n = 0; n < P; ++n) {
            bl_idx[fill[bp[n]]++] = 2 * n;
            bl_idx[fill[bq[n]]++] = 2 * n + 1;
        }
    }
    // assembly -> link CSR, link position within its assembly
    std::vector<int> al_off(NA + 1, 0), al_idx(P), link_local(P);
    for (int n = 0; n < P; ++n) al_off[h->asm_of_body[bp[n]] + 1]++;
    for (int a = 0; a < NA; ++a) al_off[a + 1] += al_off[a];
    {
        std::vector<int> fill(al_off.begin(), al_off.end() - 1);
        for (int n = 0; n < P; ++n) {
            const int a = h->asm_of_body[bp[n]];
            link_local[n] = fill[a] - al_off[a];
            al_idx[fill[a]++] = n;
        }
    }
    h->asm_link_off = al_off;
    h->asm_link_idx = al_idx;
    h->max_asm_links = 0;
    for (int a = 0; a < NA; ++a) h->max_asm_links = std::max(h->max_asm_links, al_off[a + 1] - al_off[a]);
    // connectivity: bodies of every articulated body joined by its links
    std::vector<int> parent(M);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int x) {
        while (parent[x] != x) x = parent[x] = parent[parent[x]];
        return x;
    };
    for (int n = 0; n < P; ++n) parent[find(bp[n])] = find(bq[n]);
    // An articulated body with links must be connected by them; one without
    // links (not set yet) only blocks time steps.
    h->links_connected = true;
    for (int a = 0; a < NA; ++a) {
        const int b0 = h->asm_body_idx[h->asm_body_off[a]];
        for (int k = h->asm_body_off[a]; k < h->asm_body_off[a + 1]; ++k)
            if (find(h->asm_body_idx[k]) != find(b0)) {
                h->links_connected = false;
                if (al_off[a + 1] > al_off[a])
                    return set_err(h, AM_ERR_ARG, "am_set_constraints: articulated body " + std::to_string(a) +
                                                      " is not connected by its links");
            }
    }
    // (P^a)^+ = L^+ (P^a)^T with L = (P^a)^T P^a the graph Laplacian of the
    // articulated body and L^+ = (L + J/M_a)^-1 - J/M_a (J all ones) for a
    // connected graph (Sec. 4.1, Eq. pseudo-inv-sol).  Rows follow the
    // assembly's body order, columns its link order.
    std::vector<long long> poff(NA + 1, 0);
    for (int a = 0; a < NA; ++a) {
        const long long Ma = h->asm_body_off[a + 1] - h->asm_body_off[a];
        const long long Pa = al_off[a + 1] - al_off[a];
        poff[a + 1] = poff[a] + Ma * Pa;
    }
    std::vector<double> pplus(std::max<long long>(poff[NA], 1), 0.0);
    std::vector<int> local(M);
    for (int a = 0; a < NA; ++a)
        for (int k = h->asm_body_off[a]; k < h->asm_body_off[a + 1]; ++k)
            local[h->asm_body_idx[k]] = k - h->asm_body_off[a];
    for (int a = 0; a < NA; ++a) {
        const int Ma = h->asm_body_off[a + 1] - h->asm_body_off[a];
        const int Pa = al_off[a + 1] - al_off[a];
        if (Pa == 0) continue;
        std::vector<double> Ps((size_t)Pa * Ma, 0.0);
        for (int k = 0; k < Pa; ++k) {
            const int n = al_idx[al_off[a] + k];
            Ps[(size_t)k * Ma + local[bp[n]]] += 1.0;
            Ps[(size_t)k * Ma + local[bq[n]]] -= 1.0;
        }
        std::vector<double> L((size_t)Ma * Ma, 0.0);
        for (int i = 0; i < Ma; ++i)
            for (int j = 0; j < Ma; ++j) {
                double s = 1.0 / Ma;
                for (int k = 0; k < Pa; ++k) s += Ps[(size_t)k * Ma + i] * Ps[(size_t)k * Ma + j];
                L[(size_t)i * Ma + j] = s;
            }
        if (!host_inverse(L, Ma)) return set_err(h, AM_ERR_ARG, "am_set_constraints: singular connectivity");
        for (int i = 0; i < Ma; ++i)
            for (int k = 0; k < Pa; ++k) {
                double s = 0.0;
                for (int j = 0; j < Ma; ++j) s += (L[(size_t)i * Ma + j] - 1.0 / Ma) * Ps[(size_t)k * Ma + j];
                pplus[poff[a] + (size_t)i * Pa + k] = s;
            }
    }
    // sizes of the per-assembly preconditioner and correction workspaces
    std::vector<long long> goff(NA + 1, 0), permoff(NA + 1, 0), coff(NA + 1, 0);
    for (int a = 0; a < NA; ++a) {
        const long long m = 3LL * (al_off[a + 1] - al_off[a]);
        const long long Ma = h->asm_body_off[a + 1] - h->asm_body_off[a];
        const long long nd = 7 * Ma;
        goff[a + 1] = goff[a] + m * m;
        permoff[a + 1] = permoff[a] + m;
        coff[a + 1] = coff[a] + (m ? nd * nd + 3 * nd + 3 * m : 0);
    }
    cudaStream_t s = h->stream;
    CK(dalloc(&h->d_bp, P)); CK(dalloc(&h->d_bq, P));
    CK(dalloc(&h->d_dlp, 3 * (size_t)P)); CK(dalloc(&h->d_dlq, 3 * (size_t)P));
    CK(dalloc(&h->d_dlpd, 3 * (size_t)P)); CK(dalloc(&h->d_dlqd, 3 * (size_t)P));
    CK(dalloc(&h->d_dlp1, 3 * (size_t)P)); CK(dalloc(&h->d_dlq1, 3 * (size_t)P));
    CK(dalloc(&h->d_lp, 3 * (size_t)P)); CK(dalloc(&h->d_lq, 3 * (size_t)P));
    CK(dalloc(&h->d_B, 3 * (size_t)P));
    CK(dalloc(&h->d_body_link_off, M + 1)); CK(dalloc(&h->d_body_link_idx, 2 * (size_t)P));
    CK(dalloc(&h->d_asm_link_off, NA + 1)); CK(dalloc(&h->d_asm_link_idx, P));
    CK(dalloc(&h->d_link_local, P));
    CK(dalloc(&h->d_pplus, pplus.size())); CK(dalloc(&h->d_pplus_off, NA + 1));
    const size_t esz = h->pc32 ? sizeof(float) : sizeof(double);
    CK(balloc(&h->d_G, goff[NA] * esz)); CK(balloc(&h->d_Gwork, 2 * goff[NA] * esz));
    std::vector<int> pca_asm, pca_chunk, pca_rows(NA), pca_list;
    for (int a = 0; a < NA; ++a) {
        const int m = 3 * (al_off[a + 1] - al_off[a]);
        pca_rows[a] = m;
        for (int c = 0; c * 32 < m; ++c) { pca_asm.push_back(a); pca_chunk.push_back(c); }
    }
    split_for_build(pca_rows, pca_list, h->n_pca_small, h->pca_cs);
    CK(dalloc(&h->d_pca_list, std::max(NA, 1)));
    if (NA) CK(h2d(h->d_pca_list, pca_list.data(), NA, s));
    h->n_pca = (int)pca_asm.size();
    CK(dalloc(&h->d_pca_asm, pca_asm.size())); CK(dalloc(&h->d_pca_chunk, pca_chunk.size()));
    CK(dalloc(&h->d_G_off, NA + 1)); CK(dalloc(&h->d_G_rank, NA));
    CK(dalloc(&h->d_perm, permoff[NA])); CK(dalloc(&h->d_perm_off, NA + 1));
    CK(dalloc(&h->d_corr, coff[NA])); CK(dalloc(&h->d_corr_off, NA + 1));
    CK(dalloc(&h->d_zbuf, 3 * (size_t)P)); CK(dalloc(&h->d_cbuf, 3 * (size_t)P));
    CK(h2d(h->d_bp, bp, P, s)); CK(h2d(h->d_bq, bq, P, s));
    CK(h2d(h->d_body_link_off, bl_off.data(), M + 1, s));
    CK(h2d(h->d_body_link_idx, bl_idx.data(), bl_idx.size(), s));
    CK(h2d(h->d_asm_link_off, al_off.data(), NA + 1, s));
    CK(h2d(h->d_asm_link_idx, al_idx.data(), P, s));
    CK(h2d(h->d_link_local, link_local.data(), P, s));
    CK(h2d(h->d_pplus, pplus.data(), pplus.size(), s));
    CK(h2d(h->d_pplus_off, poff.data(), NA + 1, s));
    CK(h2d(h->d_G_off, goff.data(), NA + 1, s));
    CK(h2d(h->d_perm_off, permoff.data(), NA + 1, s));
    CK(h2d(h->d_corr_off, coff.data(), NA + 1, s));
    CK(h2d(h->d_pca_asm, pca_asm.data(), pca_asm.size(), s));
    CK(h2d(h->d_pca_chunk, pca_chunk.data(), pca_chunk.size(), s));
    CK(cudaStreamSynchronize(s));
    h->n = 3 * h->Nb + 6 * h->M + 3 * P;
    h->pc_valid = false;
    return alloc_solver(h);
}

int check_quats(am_handle* h, int M, const double* theta, const char* who) {
    for (int p = 0; p < M; ++p) {
        const double* t = theta + 4 * (size_t)p;
        const double nn = std::sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2] + t[3] * t[3]);
        if (!(std::fabs(nn - 1.0) <= 1e-8))
            return set_err(h, AM_ERR_NONUNIT_QUAT, std::string(who) + ": quaternion of body " +
                                                       std::to_string(p) + " is not unit");
    }
    return AM_OK;
}

bool box_set(const am_config& c) { return c.box[0] != 0.0 || c.box[1] != 0.0 || c.box[2] != 0.0; }

int device_flags_to_status(am_handle* h, const char* who) {
    if (h->per_status) {
        const int rc = h->per_status;
        h->per_status = 0;
        return set_err(h, rc, std::string(who) + ": " + h->err);
    }
    const int f = am::take_flags(h);
    if (f & am::kFlagWall)
        return set_err(h, AM_ERR_WALL_PENETRATION, std::string(who) + ": a blob centre is at or below height a");
    if (f & am::kFlagSingular)
        return set_err(h, AM_ERR_SINGULAR, std::string(who) +
                                               ": a body's blob mobility or body mobility is not positive definite "
                                               "(bodies need at least three non-collinear blobs)");
    if (f & am::kFlagCorrection)
        return set_err(h, AM_ERR_SINGULAR, std::string(who) + ": correction normal equations not positive definite");
    if (f & am::kFlagTensor)
        return set_err(h, AM_ERR_CUDA, std::string(who) + ": a tensor-core wait of the network timed out");
    return AM_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

// pose, preconditioner and initial guess at the current configuration
int prepare(am_handle* h, const char* who, bool warm, am_step_stats* st) {
    cudaStream_t s = h->stream;
    am::launch_geometry(h);
    if (!h->sb && !h->mv_tuned && am::mobility_autotune(h))
        return set_err(h, AM_ERR_CUDA, std::string(who) + ": mobility autotuning failed");
    CK(cudaEventRecord(h->ev[0], s));
    am::pc_build(h);
    CK(cudaEventRecord(h->ev[1], s));
    CK(cudaGetLastError());
    int rc = device_flags_to_status(h, who);
    if (rc) return rc;
    if (warm && guess_from_history(h, h->t_solve, h->d_x)) {
        am::project_constraints(h, h->d_x);
    } else if (h->mlp) {
        // learned guess; with the check, per system the point on the line
        // from P~^-1 b (left in d_dx) through the learned guess with the
        // smallest residual
        if (am::learned_x0(h, h->d_x))
            return set_err(h, AM_ERR_CUDA, std::string(who) + ": learned initial guess failed");
        rc = device_flags_to_status(h, who);  // the network's tensor-core waits
        if (rc) return rc;
        const int used = h->mlp_check ? am::line_initial(h, h->d_x, h->d_dx) : h->S;
        if (st) st->learned_systems = used;
    } else {
        am::pc_apply(h, h->d_b, h->d_x);
    }
    CK(cudaGetLastError());
    if (st) st->ms_precond = elapsed(h->ev[0], h->ev[1]);
    return AM_OK;
}

int copy_outputs(am_handle* h, double* U, double* phi, double* lam) {
    cudaStream_t s = h->stream;
    if (lam) CK(d2h(lam, h->d_x, 3 * (size_t)h->Nb, s));
    if (U) CK(d2h(U, h->d_x + 3 * (size_t)h->Nb, 6 * (size_t)h->M, s));
    if (phi) CK(d2h(phi, h->d_x + 3 * (size_t)h->Nb + 6 * (size_t)h->M, 3 * (size_t)h->P, s));
    CK(cudaStreamSynchronize(s));
    return AM_OK;
}

int commit(am_handle* h, const char* who);
bool all_have_bodies(const am_handle* h);

int check_handle(am_handle* h, const char* who, bool need_bodies) {
    if (!h) { return AM_ERR_ARG; }
    if (need_bodies && h->dirty && all_have_bodies(h)) {
        const int rc = commit(h, who);
        if (rc) return rc;
    }
    if (need_bodies && !h->have_bodies) return set_err(h, AM_ERR_ARG, std::string(who) + ": no bodies set");
    return AM_OK;
}

}  // namespace

extern "C" AM_API int am_create(const am_config* cfg, am_handle** out) {
    if (!cfg || !out) return AM_ERR_ARG;
    *out = nullptr;
    am_config c = *cfg;
    if (c.restart == 0) c.restart = 50;
    if (c.max_iter == 0) c.max_iter = 500;
    if (c.corr_tol == 0.0) c.corr_tol = 1e-10;
    if (c.corr_max_iter == 0) c.corr_max_iter = 20;
    if (c.n_systems == 0) c.n_systems = 1;
    if (!(c.eta > 0.0) || !(c.blob_radius > 0.0) || (c.wall != 0 && c.wall != 1) ||
        (c.precision != AM_FP64 && c.precision != AM_MIXED) || c.n_systems < 1 || c.n_systems > 65536 ||
        !(c.tol > 0.0) ||
        c.restart < 1 || c.restart > 200 || c.max_iter < 1 || !(c.corr_tol > 0.0) || c.corr_max_iter < 1 ||
        (c.single_blob != 0 && c.single_blob != 1) ||
        (c.single_blob && (c.wall || c.precision != AM_FP64)))
        return AM_ERR_ARG;
    if (box_set(c)) {
        // periodic box: every side positive and finite; free space, one
        // system of multi-blob bodies
        for (int d = 0; d < 3; ++d)
            if (!(c.box[d] > 0.0) || !std::isfinite(c.box[d])) return AM_ERR_ARG;
        if (c.wall || c.single_blob || c.n_systems != 1) return AM_ERR_ARG;
        if (c.ewald_tol == 0.0) c.ewald_tol = 1e-10;
        if (!(c.ewald_tol >= 1e-14 && c.ewald_tol <= 1e-3) || !(c.ewald_xi >= 0.0) || !std::isfinite(c.ewald_xi))
            return AM_ERR_ARG;
    }
    am_handle* h = new am_handle();
    h->cfg = c;
    h->restart = c.restart;
    h->pc32 = (c.precision == AM_MIXED);
    h->sb = c.single_blob != 0;
    h->S = c.n_systems;
    h->sys.resize(h->S);
    h->prm = am::make_params(c.eta, c.blob_radius);
    if (c.cuda_stream) {
        h->stream = static_cast<cudaStream_t>(c.cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return AM_ERR_CUDA;
        }
        h->own_stream = true;
    }
    bool ok = cudaMallocHost(reinterpret_cast<void**>(&h->h_scal), 32 * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(reinterpret_cast<void**>(&h->h_flags), sizeof(int)) == cudaSuccess &&
              cudaMalloc(reinterpret_cast<void**>(&h->d_scal), 32 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(reinterpret_cast<void**>(&h->d_flags), sizeof(int)) == cudaSuccess &&
              cudaMalloc(reinterpret_cast<void**>(&h->d_red), 4 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(reinterpret_cast<void**>(&h->d_ctrl), sizeof(am::ArnoldiCtrl)) == cudaSuccess &&
              cudaMallocHost(reinterpret_cast<void**>(&h->h_ctrl), sizeof(am::ArnoldiCtrl)) == cudaSuccess &&
              cudaMemset(h->d_flags, 0, sizeof(int)) == cudaSuccess;
    for (int k = 0; k < 8 && ok; ++k) ok = cudaEventCreate(&h->ev[k]) == cudaSuccess;
    if (!ok) {
        am_destroy(h);
        return AM_ERR_CUDA;
    }
    *out = h;
    return AM_OK;
}

namespace {

// Checks one system's bodies; returns its articulated-body count and largest
// body (blobs).
int validate_bodies(am_handle* h, int M, const double* q, const double* theta, const int* blob_offset,
                    const double* rho, const double* F, const int* asm_of_body, int* NA_out, int* maxb_out) {
    const char* who = "am_set_bodies";
    if (M <= 0 || !q || !theta || !blob_offset || !rho || !F || !asm_of_body)
        return set_err(h, AM_ERR_ARG, "am_set_bodies: n_bodies <= 0 or NULL array");
    if (blob_offset[0] != 0) return set_err(h, AM_ERR_ARG, "am_set_bodies: blob_offset[0] != 0");
    int maxb = 0;
    for (int p = 0; p < M && !h->sb; ++p) {
        const int c = blob_offset[p + 1] - blob_offset[p];
        if (c < 1) return set_err(h, AM_ERR_ARG, "am_set_bodies: body without blobs");
        maxb = std::max(maxb, c);
    }
    if ((size_t)3 * maxb * (h->pc32 ? 4 : 8) > 200 * 1024)
        return set_err(h, AM_ERR_ARG, "am_set_bodies: a body has more blobs than the preconditioner "
                                      "build supports (8,533 in FP64, 17,066 in mixed precision)");
    if (blob_offset[M] > (1 << 28)) return set_err(h, AM_ERR_ARG, "am_set_bodies: too many blobs");
    int NA = 0;
    for (int p = 0; p < M; ++p) {
        if (asm_of_body[p] < 0 || asm_of_body[p] >= M)
            return set_err(h, AM_ERR_ARG, "am_set_bodies: assembly index out of range");
        NA = std::max(NA, asm_of_body[p] + 1);
    }
    std::vector<int> cnt(NA, 0);
    for (int p = 0; p < M; ++p) cnt[asm_of_body[p]]++;
    for (int a = 0; a < NA; ++a)
        if (!cnt[a]) return set_err(h, AM_ERR_ARG, "am_set_bodies: unused assembly index");
    int rc = check_quats(h, M, theta, who);
    if (rc) return rc;
    *NA_out = NA;
    *maxb_out = maxb;
    return AM_OK;
}

// Device layout of the bodies of all systems (concatenated arrays).
int build_layout(am_handle* h, int M, int Nb, int NA, int maxb, const double* q, const double* theta,
                 const int* blob_offset, const double* rho, const double* F, const double* slip,
                 const int* asm_of_body) {
    std::vector<int> cnt(NA, 0);
    for (int p = 0; p < M; ++p) cnt[asm_of_body[p]]++;
    free_links(h);
    free_bodies(h);
    free_solver(h);
    h->have_bodies = false;
    h->M = M;
    h->Nb = Nb;
    h->NA = NA;
    h->P = 0;
    h->max_body_blobs = maxb;
    h->blob_off.assign(blob_offset, blob_offset + M + 1);
    h->asm_of_body.assign(asm_of_body, asm_of_body + M);
    h->asm_body_off.assign(NA + 1, 0);
    for (int a = 0; a < NA; ++a) h->asm_body_off[a + 1] = h->asm_body_off[a] + cnt[a];
    h->asm_body_idx.assign(M, 0);
    std::vector<int> body_local(M);
    {
        std::vector<int> fill(h->asm_body_off.begin(), h->asm_body_off.end() - 1);
        for (int p = 0; p < M; ++p) {
            const int a = asm_of_body[p];
            body_local[p] = fill[a] - h->asm_body_off[a];
            h->asm_body_idx[fill[a]++] = p;
        }
    }
    std::vector<int> body_of_blob(Nb);
    std::vector<long long> moff(M + 1, 0);
    for (int p = 0; p < M; ++p) {
        for (int i = blob_offset[p]; i < blob_offset[p + 1]; ++i) body_of_blob[i] = p;
        const long long m = 3LL * (blob_offset[p + 1] - blob_offset[p]);
        moff[p + 1] = moff[p] + m * m;
    }
    h->minv_total = moff[M];
    cudaStream_t s = h->stream;
    CK(dalloc(&h->d_q, 3 * (size_t)M)); CK(dalloc(&h->d_theta, 4 * (size_t)M));
    CK(dalloc(&h->d_rho, 3 * (size_t)Nb)); CK(dalloc(&h->d_F, 6 * (size_t)M));
    if (slip) CK(dalloc(&h->d_slip, 3 * (size_t)Nb));
    CK(dalloc(&h->d_blob_off, M + 1)); CK(dalloc(&h->d_body_of_blob, Nb));
    CK(dalloc(&h->d_asm_of_body, M)); CK(dalloc(&h->d_asm_body_off, NA + 1));
    CK(dalloc(&h->d_asm_body_idx, M)); CK(dalloc(&h->d_body_local, M));
    CK(dalloc(&h->d_r4, Nb)); CK(dalloc(&h->d_d4, Nb)); CK(dalloc(&h->d_rhi, Nb));
    CK(dalloc(&h->d_rlo, Nb)); CK(dalloc(&h->d_r3, 3 * (size_t)Nb));
    const size_t esz = h->pc32 ? sizeof(float) : sizeof(double);
    CK(balloc(&h->d_minv, h->minv_total * esz)); CK(balloc(&h->d_pcwork, 2 * h->minv_total * esz));
    CK(balloc(&h->d_Y, 18 * (size_t)Nb * esz)); CK(dalloc(&h->d_Nt, 36 * (size_t)M));
    std::vector<int> pcw_body, pcw_chunk, pcw_off(M + 1, 0);
    for (int p = 0; p < M; ++p) {
        const int m = 3 * (blob_offset[p + 1] - blob_offset[p]);
        for (int c = 0; c * 32 < m; ++c) { pcw_body.push_back(p); pcw_chunk.push_back(c); }
        pcw_off[p + 1] = (int)pcw_body.size();
    }
    h->n_pcw = (int)pcw_body.size();
    std::vector<int> pcb_rows(M), pcb_list;
    for (int p = 0; p < M; ++p) pcb_rows[p] = 3 * (blob_offset[p + 1] - blob_offset[p]);
    split_for_build(pcb_rows, pcb_list, h->n_pcb_small, h->pcb_cs);
    CK(dalloc(&h->d_pcb_list, std::max(M, 1)));
    CK(dalloc(&h->d_pcw_body, pcw_body.size())); CK(dalloc(&h->d_pcw_chunk, pcw_chunk.size()));
    CK(dalloc(&h->d_pcw_off, M + 1)); CK(dalloc(&h->d_ytp, 6 * pcw_body.size()));
    CK(dalloc(&h->d_pcb_cnt, M));
    CK(cudaMemsetAsync(h->d_pcb_cnt, 0, std::max(M, 1) * sizeof(int), s));
    CK(dalloc(&h->d_minv_off, M + 1)); CK(dalloc(&h->d_pc_w, 3 * (size_t)Nb));
    CK(dalloc(&h->d_pc_Uhat, 6 * (size_t)M));
    CK(dalloc(&h->d_qnew, 3 * (size_t)M)); CK(dalloc(&h->d_thnew, 4 * (size_t)M));
    CK(dalloc(&h->d_q0, 3 * (size_t)M)); CK(dalloc(&h->d_th0, 4 * (size_t)M));
    CK(dalloc(&h->d_fst, 3 * (size_t)Nb));
    if (h->sb) CK(dalloc(&h->d_sbpart, (size_t)am::kSbChunks * 6 * M));
    CK(dalloc(&h->d_iters, NA));
    if (h->h_iters) cudaFreeHost(h->h_iters);
    h->h_iters = nullptr;
    CK(cudaMallocHost(reinterpret_cast<void**>(&h->h_iters), std::max(NA, 1) * sizeof(int)));
    CK(h2d(h->d_q, q, 3 * (size_t)M, s)); CK(h2d(h->d_theta, theta, 4 * (size_t)M, s));
    CK(h2d(h->d_rho, rho, 3 * (size_t)Nb, s)); CK(h2d(h->d_F, F, 6 * (size_t)M, s));
    if (slip) CK(h2d(h->d_slip, slip, 3 * (size_t)Nb, s));
    CK(h2d(h->d_blob_off, blob_offset, M + 1, s));
    CK(h2d(h->d_body_of_blob, body_of_blob.data(), Nb, s));
    CK(h2d(h->d_asm_of_body, asm_of_body, M, s));
    CK(h2d(h->d_asm_body_off, h->asm_body_off.data(), NA + 1, s));
    CK(h2d(h->d_asm_body_idx, h->asm_body_idx.data(), M, s));
    CK(h2d(h->d_body_local, body_local.data(), M, s));
    CK(h2d(h->d_minv_off, moff.data(), M + 1, s));
    if (M) CK(h2d(h->d_pcb_list, pcb_list.data(), M, s));
    CK(h2d(h->d_pcw_body, pcw_body.data(), pcw_body.size(), s));
    CK(h2d(h->d_pcw_chunk, pcw_chunk.data(), pcw_chunk.size(), s));
    CK(h2d(h->d_pcw_off, pcw_off.data(), M + 1, s));
    CK(cudaStreamSynchronize(s));
    return AM_OK;
}

// Per-system maps of the batched solve: system of every unknown, dot-product
// chunks that never straddle two systems (listed system by system), the
// per-system GMRES scalars and the mobility bookkeeping.
int build_system_maps(am_handle* h) {
    const int S = h->S, n = h->n, m = h->restart;
    std::vector<int> sys_of_elem(n), sys_of_blob(h->Nb);
    std::vector<int> cs, ce, coff(S + 1, 0);
    const int nl = 3 * h->Nb, nu = 6 * h->M;
    // Chunk length: about n / (4 x SMs), rounded up to a power of two in
    // 64 .. 1024, so that the FP64 dot products and orthogonalisation of a
    // small system still spread over all SMs (GB300 has 2 FP64 FMAs per SM
    // per cycle); the chunk kernels run 256 threads a block.
    const long long per = ((long long)n + 4LL * am::num_sms() - 1) / (4LL * am::num_sms());
    int clen = 64;
    while (clen < per && clen < 1024) clen *= 2;
    h->chunk_len = clen;
    h->chunk_threads = 256;
    for (int sI = 0; sI < S; ++sI) {
        const am_sys_rec& r = h->sys[sI];
        const int segs[3][2] = {{3 * h->sys_blob0[sI], 3 * (h->sys_blob0[sI] + r.Nb)},
                                {nl + 6 * h->sys_body0[sI], nl + 6 * (h->sys_body0[sI] + r.M)},
                                {nl + nu + 3 * h->sys_link0[sI], nl + nu + 3 * (h->sys_link0[sI] + r.P)}};
        for (auto& sg : segs) {
            for (int i = sg[0]; i < sg[1]; ++i) sys_of_elem[i] = sI;
            for (int c0 = sg[0]; c0 < sg[1]; c0 += clen) {
                cs.push_back(c0);
                ce.push_back(std::min(sg[1], c0 + clen));
            }
        }
        for (int i = 0; i < r.Nb; ++i) sys_of_blob[h->sys_blob0[sI] + i] = sI;
        coff[sI + 1] = (int)cs.size();
    }
    h->nchunks = (int)cs.size();
    cudaStream_t st = h->stream;
    CK(dalloc(&h->d_sys_of_elem, n)); CK(dalloc(&h->d_sys_of_blob, h->Nb));
    CK(dalloc(&h->d_chunk_start, cs.size())); CK(dalloc(&h->d_chunk_end, ce.size()));
    CK(dalloc(&h->d_sys_chunk_off, S + 1));
    CK(dalloc(&h->d_Hs, (size_t)S * (m + 1) * m)); CK(dalloc(&h->d_css, (size_t)S * m));
    CK(dalloc(&h->d_sns, (size_t)S * m)); CK(dalloc(&h->d_gs, (size_t)S * (m + 1)));
    CK(dalloc(&h->d_coefs, (size_t)S * (m + 1))); CK(dalloc(&h->d_xis, (size_t)S * (m + 1)));
    CK(dalloc(&h->d_hcols, (size_t)S * (m + 1)));
    CK(dalloc(&h->d_bnorm_s, S)); CK(dalloc(&h->d_beta_s, S)); CK(dalloc(&h->d_inv_s, S));
    CK(dalloc(&h->d_tol_s, S)); CK(dalloc(&h->d_sysred, 4 * (size_t)S + 16));
    CK(dalloc(&h->d_active, S)); CK(dalloc(&h->d_kdone, S));
    CK(dalloc(&h->d_arn_cnt, S + 1));
    CK(cudaMemsetAsync(h->d_arn_cnt, 0, (S + 1) * sizeof(int), st));
    CK(dalloc(&h->d_part, (size_t)(m + 1) * std::max(1, h->nchunks)));
    CK(dalloc(&h->d_npart, std::max(h->nchunks, 4 * am::num_sms() + 64)));
    std::vector<int> b0(S), nb(S), bo(S + 1, h->M);
    for (int sI = 0; sI < S; ++sI) { b0[sI] = h->sys_blob0[sI]; nb[sI] = h->sys[sI].Nb; bo[sI] = h->sys_body0[sI]; }
    CK(dalloc(&h->d_sys_body_off, S + 1));
    CK(h2d(h->d_sys_body_off, bo.data(), S + 1, st));
    CK(dalloc(&h->d_sys_blob0, S)); CK(dalloc(&h->d_sys_nb, S));
    CK(dalloc(&h->d_sys_nch, S)); CK(dalloc(&h->d_sys_poff, S));
    CK(dalloc(&h->d_item_counter, 2));  // work queue: next item, blocks finished (both start at 0)
    CK(cudaMemsetAsync(h->d_item_counter, 0, 2 * sizeof(int), st));
    CK(h2d(h->d_sys_of_elem, sys_of_elem.data(), n, st));
    CK(h2d(h->d_sys_of_blob, sys_of_blob.data(), h->Nb, st));
    CK(h2d(h->d_chunk_start, cs.data(), cs.size(), st));
    CK(h2d(h->d_chunk_end, ce.data(), ce.size(), st));
    CK(h2d(h->d_sys_chunk_off, coff.data(), S + 1, st));
    CK(h2d(h->d_sys_blob0, b0.data(), S, st));
    CK(h2d(h->d_sys_nb, nb.data(), S, st));
    CK(cudaStreamSynchronize(st));
    h->mv_tuned = false;
    if (box_set(h->cfg)) {
        const int rc = am::periodic_setup(h);
        if (rc) return set_err(h, rc, "am_set_bodies: " + h->err);
    }
    return am::mobility_layout(h, h->cfg.precision == AM_MIXED ? 2 : 1, 0) ? AM_ERR_CUDA : AM_OK;
}

bool all_have_bodies(const am_handle* h) {
    for (const auto& r : h->sys)
        if (!r.has_bodies) return false;
    return true;
}

// Copies the device state (positions, orientations, link vectors, which
// steps advance) back into the records before they are rebuilt.
int sync_records(am_handle* h) {
    if (!h->committed || h->dirty) return AM_OK;
    std::vector<double> q(3 * (size_t)h->M), th(4 * (size_t)h->M), dlp(3 * (size_t)h->P), dlq(3 * (size_t)h->P);
    cudaStream_t s = h->stream;
    CK(d2h(q.data(), h->d_q, q.size(), s));
    CK(d2h(th.data(), h->d_theta, th.size(), s));
    if (h->P) {
        CK(d2h(dlp.data(), h->d_dlp, dlp.size(), s));
        CK(d2h(dlq.data(), h->d_dlq, dlq.size(), s));
    }
    CK(cudaStreamSynchronize(s));
    for (int sI = 0; sI < h->S; ++sI) {
        am_sys_rec& r = h->sys[sI];
        const int b0 = h->sys_body0[sI], l0 = h->sys_link0[sI];
        std::copy(q.begin() + 3 * b0, q.begin() + 3 * (b0 + r.M), r.q.begin());
        std::copy(th.begin() + 4 * b0, th.begin() + 4 * (b0 + r.M), r.theta.begin());
        if (r.P) {
            std::copy(dlp.begin() + 3 * l0, dlp.begin() + 3 * (l0 + r.P), r.dlp.begin());
            std::copy(dlq.begin() + 3 * l0, dlq.begin() + 3 * (l0 + r.P), r.dlq.begin());
        }
    }
    return AM_OK;
}

// Builds the device layout of all systems from the records.
int commit(am_handle* h, const char* who) {
    if (!h->dirty && h->committed) return AM_OK;
    if (!all_have_bodies(h)) return set_err(h, AM_ERR_ARG, std::string(who) + ": some system has no bodies");
    const int S = h->S;
    h->sys_body0.assign(S, 0); h->sys_blob0.assign(S, 0); h->sys_link0.assign(S, 0); h->sys_asm0.assign(S, 0);
    int M = 0, Nb = 0, NA = 0, P = 0, maxb = 0;
    bool any_slip = false, any_active = false;
    for (int sI = 0; sI < S; ++sI) {
        const am_sys_rec& r = h->sys[sI];
        h->sys_body0[sI] = M; h->sys_blob0[sI] = Nb; h->sys_link0[sI] = P; h->sys_asm0[sI] = NA;
        M += r.M; Nb += r.Nb; NA += r.NA; P += r.P;
        for (int p = 0; p < r.M; ++p) maxb = std::max(maxb, r.blob_off[p + 1] - r.blob_off[p]);
        any_slip |= !r.slip.empty();
        any_active |= !r.dlpd.empty();
    }
    std::vector<double> q, th, rho, F, slip, dlp, dlq, dlpd, dlqd;
    std::vector<int> off(1, 0), asmb, bp, bq;
    for (int sI = 0; sI < S; ++sI) {
        const am_sys_rec& r = h->sys[sI];
        q.insert(q.end(), r.q.begin(), r.q.end());
        th.insert(th.end(), r.theta.begin(), r.theta.end());
        rho.insert(rho.end(), r.rho.begin(), r.rho.end());
        F.insert(F.end(), r.F.begin(), r.F.end());
        if (any_slip) {
            if (r.slip.empty()) slip.insert(slip.end(), 3 * (size_t)r.Nb, 0.0);
            else slip.insert(slip.end(), r.slip.begin(), r.slip.end());
        }
        for (int p = 0; p < r.M; ++p) {
            off.push_back(h->sys_blob0[sI] + r.blob_off[p + 1]);
            asmb.push_back(h->sys_asm0[sI] + r.asm_of_body[p]);
        }
        for (int k = 0; k < r.P; ++k) {
            bp.push_back(h->sys_body0[sI] + r.bp[k]);
            bq.push_back(h->sys_body0[sI] + r.bq[k]);
        }
        dlp.insert(dlp.end(), r.dlp.begin(), r.dlp.end());
        dlq.insert(dlq.end(), r.dlq.begin(), r.dlq.end());
        if (r.dlpd.empty()) {
            dlpd.insert(dlpd.end(), 3 * (size_t)r.P, 0.0);
            dlqd.insert(dlqd.end(), 3 * (size_t)r.P, 0.0);
        } else {
            dlpd.insert(dlpd.end(), r.dlpd.begin(), r.dlpd.end());
            dlqd.insert(dlqd.end(), r.dlqd.begin(), r.dlqd.end());
        }
    }
    h->committed = false;
    int rc = build_layout(h, M, Nb, NA, maxb, q.data(), th.data(), off.data(), rho.data(), F.data(),
                          any_slip ? slip.data() : nullptr, asmb.data());
    if (rc) return rc;
    rc = build_links(h, P, bp.data(), bq.data());
    if (rc) return rc;
    cudaStream_t s = h->stream;
    CK(h2d(h->d_dlp, dlp.data(), dlp.size(), s));
    CK(h2d(h->d_dlq, dlq.data(), dlq.size(), s));
    CK(h2d(h->d_dlpd, dlpd.data(), dlpd.size(), s));
    CK(h2d(h->d_dlqd, dlqd.data(), dlqd.size(), s));
    CK(cudaStreamSynchronize(s));
    h->active_links = any_active;
    rc = build_system_maps(h);
    if (rc) return set_err(h, rc, std::string(who) + ": device allocation failed");
    h->have_bodies = true;
    h->committed = true;
    h->dirty = false;
    am::launch_geometry(h);
    CK(cudaGetLastError());
    rc = device_flags_to_status(h, who);
    if (rc) {
        h->have_bodies = false;
        h->committed = false;
        h->dirty = true;
        return rc;
    }
    return AM_OK;
}

int check_system(am_handle* h, int system, const char* who) {
    if (system < 0 || system >= h->S) return set_err(h, AM_ERR_ARG, std::string(who) + ": system out of range");
    return AM_OK;
}

}  // namespace

extern "C" AM_API int am_set_bodies(am_handle* h, int system, int M, const double* q, const double* theta,
                                    const int* blob_offset, const double* rho, const double* F,
                                    const double* slip, const int* asm_of_body) {
    if (!h) return AM_ERR_ARG;
    int rc = check_system(h, system, "am_set_bodies");
    if (rc) return rc;
    int NA = 0, maxb = 0;
    // single-blob bodies carry no blobs of their own: the body is the blob
    std::vector<int> no_blobs;
    static const double no_rho = 0.0;
    if (h->sb && M > 0) {
        no_blobs.assign(M + 1, 0);
        blob_offset = no_blobs.data();
        rho = &no_rho;
        slip = nullptr;
    }
    rc = validate_bodies(h, M, q, theta, blob_offset, rho, F, asm_of_body, &NA, &maxb);
    if (rc) return rc;
    rc = sync_records(h);
    if (rc) return rc;
    am_sys_rec& r = h->sys[system];
    const int Nb = blob_offset[M];
    r.has_bodies = true;
    r.M = M; r.Nb = Nb; r.NA = NA; r.P = 0;
    r.q.assign(q, q + 3 * (size_t)M);
    r.theta.assign(theta, theta + 4 * (size_t)M);
    r.rho.assign(rho, rho + 3 * (size_t)Nb);
    r.F.assign(F, F + 6 * (size_t)M);
    if (slip) r.slip.assign(slip, slip + 3 * (size_t)Nb); else r.slip.clear();
    r.blob_off.assign(blob_offset, blob_offset + M + 1);
    r.asm_of_body.assign(asm_of_body, asm_of_body + M);
    r.bp.clear(); r.bq.clear(); r.dlp.clear(); r.dlq.clear(); r.dlpd.clear(); r.dlqd.clear();
    h->dirty = true;
    h->have_bodies = false;
    // one system: build the device layout now (errors surface here); several:
    // on first use, so that loading S systems does not rebuild S times
    if (h->S == 1) return commit(h, "am_set_bodies");
    return AM_OK;
}

extern "C" AM_API int am_set_constraints(am_handle* h, int system, int P, const int* bp, const int* bq,
                                         const double* dlp, const double* dlq, const double* dlpd,
                                         const double* dlqd) {
    if (!h) return AM_ERR_ARG;
    int rc = check_system(h, system, "am_set_constraints");
    if (rc) return rc;
    am_sys_rec& r = h->sys[system];
    if (!r.has_bodies) return set_err(h, AM_ERR_ARG, "am_set_constraints: no bodies set for this system");
    if (P < 0 || (P > 0 && (!bp || !bq || !dlp || !dlq)))
        return set_err(h, AM_ERR_ARG, "am_set_constraints: n_links < 0 or NULL array");
    if ((dlpd == nullptr) != (dlqd == nullptr))
        return set_err(h, AM_ERR_ARG, "am_set_constraints: give both link derivatives or neither");
    for (int n = 0; n < P; ++n) {
        if (bp[n] < 0 || bp[n] >= r.M || bq[n] < 0 || bq[n] >= r.M)
            return set_err(h, AM_ERR_ARG, "am_set_constraints: body index out of range");
        if (bp[n] == bq[n]) return set_err(h, AM_ERR_ARG, "am_set_constraints: link joins a body to itself");
        if (r.asm_of_body[bp[n]] != r.asm_of_body[bq[n]])
            return set_err(h, AM_ERR_ARG, "am_set_constraints: link joins two articulated bodies");
    }
    const bool same = h->committed && !h->dirty && P == r.P && std::equal(bp, bp + P, r.bp.begin()) &&
                      std::equal(bq, bq + P, r.bq.begin());
    if (!same) {
        rc = sync_records(h);
        if (rc) return rc;
    }
    r.P = P;
    r.bp.assign(bp, bp + P); r.bq.assign(bq, bq + P);
    r.dlp.assign(dlp, dlp + 3 * (size_t)P); r.dlq.assign(dlq, dlq + 3 * (size_t)P);
    if (dlpd) {
        r.dlpd.assign(dlpd, dlpd + 3 * (size_t)P);
        r.dlqd.assign(dlqd, dlqd + 3 * (size_t)P);
    } else {
        r.dlpd.clear(); r.dlqd.clear();
    }
    if (!same) {
        h->dirty = true;
        h->have_bodies = false;
        if (h->S == 1) return commit(h, "am_set_constraints");
        return AM_OK;
    }
    // same connectivity: update this system's link vectors in place
    cudaStream_t s = h->stream;
    const size_t o = 3 * (size_t)h->sys_link0[system];
    CK(h2d(h->d_dlp + o, dlp, 3 * (size_t)P, s));
    CK(h2d(h->d_dlq + o, dlq, 3 * (size_t)P, s));
    if (dlpd) {
        CK(h2d(h->d_dlpd + o, dlpd, 3 * (size_t)P, s));
        CK(h2d(h->d_dlqd + o, dlqd, 3 * (size_t)P, s));
    } else if (P) {
        CK(cudaMemsetAsync(h->d_dlpd + o, 0, 3 * (size_t)P * sizeof(double), s));
        CK(cudaMemsetAsync(h->d_dlqd + o, 0, 3 * (size_t)P * sizeof(double), s));
    }
    CK(cudaStreamSynchronize(s));
    bool any_active = false;
    for (const auto& rr : h->sys) any_active |= !rr.dlpd.empty();
    h->active_links = any_active;
    h->pc_valid = false;
    return AM_OK;
}

extern "C" AM_API int am_set_joints(am_handle* h, int system, int P, const int* bp, const int* bq,
                                    const double* joint) {
    if (!h) return AM_ERR_ARG;
    int rc = check_system(h, system, "am_set_joints");
    if (rc) return rc;
    am_sys_rec& r = h->sys[system];
    if (!r.has_bodies) return set_err(h, AM_ERR_ARG, "am_set_joints: no bodies set for this system");
    if (P < 0 || (P > 0 && (!bp || !bq || !joint)))
        return set_err(h, AM_ERR_ARG, "am_set_joints: n_links < 0 or NULL array");
    rc = sync_records(h);
    if (rc) return rc;
    const std::vector<double>& q = r.q;
    const std::vector<double>& th = r.theta;
    std::vector<double> dlp(3 * (size_t)P), dlq(3 * (size_t)P);
    for (int n = 0; n < P; ++n) {
        if (bp[n] < 0 || bp[n] >= r.M || bq[n] < 0 || bq[n] >= r.M)
            return set_err(h, AM_ERR_ARG, "am_set_joints: body index out of range");
        double v[3];
        for (int a = 0; a < 3; ++a) v[a] = joint[3 * n + a] - q[3 * bp[n] + a];
        host_rotate(&th[4 * bp[n]], v, &dlp[3 * n], true);
        for (int a = 0; a < 3; ++a) v[a] = joint[3 * n + a] - q[3 * bq[n] + a];
        host_rotate(&th[4 * bq[n]], v, &dlq[3 * n], true);
    }
    return am_set_constraints(h, system, P, bp, bq, dlp.data(), dlq.data(), nullptr, nullptr);
}

extern "C" AM_API int am_solve(am_handle* h, am_step_stats* stats, double* U, double* phi, double* lam) {
    if (!h) return AM_ERR_ARG;
    am_step_stats st{};
    int rc = check_handle(h, "am_solve", true);
    if (rc) return rc;
    const long long l0 = am::g_launches.load();
    h->pairs = 0;
    rc = prepare(h, "am_solve", false, &st);
    if (rc) return rc;
    CK(cudaEventRecord(h->ev[2], h->stream));
    rc = am::solve(h, &st);
    CK(cudaEventRecord(h->ev[3], h->stream));
    CK(cudaGetLastError());
    int rc2 = copy_outputs(h, U, phi, lam);
    if (rc2) return rc2;
    st.ms_gmres = elapsed(h->ev[2], h->ev[3]);
    st.pairs = h->pairs;
    st.kernel_launches = (int)(am::g_launches.load() - l0);
    st.status = rc;
    if (stats) *stats = st;
    if (rc == AM_ERR_NOT_CONVERGED) set_err(h, rc, "am_solve: GMRES did not reach the tolerance");
    return rc;
}

extern "C" AM_API int am_learned_features(am_handle* h, float* X, float* T) {
    if (!h) return AM_ERR_ARG;
    if (!X) return set_err(h, AM_ERR_ARG, "am_learned_features: NULL feature array");
    if (box_set(h->cfg)) return set_err(h, AM_ERR_ARG, "am_learned_features: not for a periodic box");
    int rc = check_handle(h, "am_learned_features", true);
    if (rc) return rc;
    am::launch_geometry(h);
    am::pc_build(h);
    CK(cudaGetLastError());
    rc = device_flags_to_status(h, "am_learned_features");
    if (rc) return rc;
    if (am::learned_features(h, X, T)) return set_err(h, AM_ERR_CUDA, "am_learned_features: kernel failed");
    return AM_OK;
}

extern "C" AM_API int am_set_initial_guess(am_handle* h, int order) {
    if (!h) return AM_ERR_ARG;
    if (order < 0 || order > 3) return set_err(h, AM_ERR_ARG, "am_set_initial_guess: order must be 0..3");
    h->guess_order = order;
    return AM_OK;
}

extern "C" AM_API int am_set_learned(am_handle* h, am_mlp* model, int check) {
    if (!h) return AM_ERR_ARG;
    if (h->sb && model) return set_err(h, AM_ERR_ARG, "am_set_learned: not for single-blob bodies");
    if (box_set(h->cfg) && model) return set_err(h, AM_ERR_ARG, "am_set_learned: not for a periodic box");
    h->mlp = model;
    h->mlp_check = check != 0;
    return AM_OK;
}

extern "C" AM_API int am_solve_step(am_handle* h, double t, double dt, const double* dlp_next,
                                    const double* dlq_next, am_step_stats* stats, double* U, double* phi,
                                    double* lam) {
    if (!h) return AM_ERR_ARG;
    am_step_stats st{};
    int rc = check_handle(h, "am_solve_step", true);
    if (rc) return rc;
    if (!(dt > 0.0) || !std::isfinite(dt)) return set_err(h, AM_ERR_ARG, "am_solve_step: dt must be > 0");
    if ((dlp_next == nullptr) != (dlq_next == nullptr))
        return set_err(h, AM_ERR_ARG, "am_solve_step: give both next link vectors or neither");
    if (!h->links_connected)
        return set_err(h, AM_ERR_ARG, "am_solve_step: an articulated body of several bodies has no links "
                                      "joining them (set them with am_set_constraints)");
    const long long l0 = am::g_launches.load();
    h->pairs = 0;
    cudaStream_t s = h->stream;
    h->t_solve = t;
    rc = prepare(h, "am_solve_step", true, &st);
    if (rc) return rc;
    CK(cudaEventRecord(h->ev[2], s));
    int rs = am::solve(h, &st);
    CK(cudaEventRecord(h->ev[3], s));
    CK(cudaGetLastError());
    rc = copy_outputs(h, U, phi, lam);
    if (rc) return rc;
    push_history(h, t, h->d_x);
    CK(cudaGetLastError());
    if (h->P) {
        if (dlp_next) {
            CK(h2d(h->d_dlp1, dlp_next, 3 * (size_t)h->P, s));
            CK(h2d(h->d_dlq1, dlq_next, 3 * (size_t)h->P, s));
        } else {
            CK(cudaMemcpyAsync(h->d_dlp1, h->d_dlp, 3 * h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(h->d_dlq1, h->d_dlq, 3 * h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
    }
    CK(cudaEventRecord(h->ev[4], s));
    rc = am::advance(h, dt, &st);
    CK(cudaEventRecord(h->ev[5], s));
    CK(cudaGetLastError());
    if (rc) return rc;
    rc = device_flags_to_status(h, "am_solve_step");
    if (rc) return rc;
    CK(cudaStreamSynchronize(s));
    st.ms_gmres = elapsed(h->ev[2], h->ev[3]);
    st.ms_update = elapsed(h->ev[4], h->ev[5]);
    st.pairs = h->pairs;
    st.kernel_launches = (int)(am::g_launches.load() - l0);
    st.status = rs;
    h->pc_valid = false;
    if (stats) *stats = st;
    if (rs == AM_ERR_NOT_CONVERGED) set_err(h, rs, "am_solve_step: GMRES did not reach the tolerance");
    return rs;
}

// Link vectors at the end of a (half) step into d_dlp1/d_dlq1: the given
// host arrays, or the current ones.
static int set_end_links(am_handle* h, const double* dlp, const double* dlq) {
    if (!h->P) return AM_OK;
    cudaStream_t s = h->stream;
    if (dlp) {
        CK(h2d(h->d_dlp1, dlp, 3 * (size_t)h->P, s));
        CK(h2d(h->d_dlq1, dlq, 3 * (size_t)h->P, s));
    } else {
        CK(cudaMemcpyAsync(h->d_dlp1, h->d_dlp, 3 * h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(h->d_dlq1, h->d_dlq, 3 * h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    return AM_OK;
}

// One solve at the current pose at time t (guess from the history) with its
// timings into st.
static int stage_solve(am_handle* h, const char* who, double t, am_step_stats* st, int* rs) {
    cudaStream_t s = h->stream;
    h->t_solve = t;
    int rc = prepare(h, who, true, st);
    if (rc) return rc;
    CK(cudaEventRecord(h->ev[2], s));
    *rs = am::solve(h, st);
    CK(cudaEventRecord(h->ev[3], s));
    CK(cudaGetLastError());
    push_history(h, t, h->d_x);
    CK(cudaGetLastError());
    CK(cudaEventSynchronize(h->ev[3]));
    st->ms_gmres = elapsed(h->ev[2], h->ev[3]);
    return AM_OK;
}

extern "C" AM_API int am_solve_step_rk2(am_handle* h, double t, double dt, const double* dlp_half,
                                        const double* dlq_half, const double* dlpd_half,
                                        const double* dlqd_half, const double* dlp_next,
                                        const double* dlq_next, am_step_stats* stats, double* U, double* phi,
                                        double* lam) {
    const char* who = "am_solve_step_rk2";
    if (!h) return AM_ERR_ARG;
    int rc = check_handle(h, who, true);
    if (rc) return rc;
    if (!(dt > 0.0) || !std::isfinite(dt)) return set_err(h, AM_ERR_ARG, std::string(who) + ": dt must be > 0");
    if ((dlp_half == nullptr) != (dlq_half == nullptr) || (dlp_next == nullptr) != (dlq_next == nullptr) ||
        (dlpd_half == nullptr) != (dlqd_half == nullptr))
        return set_err(h, AM_ERR_ARG, std::string(who) + ": give both link arrays of a pair or neither");
    if (h->P && h->active_links && !dlpd_half)
        return set_err(h, AM_ERR_ARG, std::string(who) + ": active links need their derivatives at the midpoint");
    if (!h->active_links && dlpd_half)
        return set_err(h, AM_ERR_ARG, std::string(who) + ": passive links take no derivatives");
    if (!h->links_connected)
        return set_err(h, AM_ERR_ARG, std::string(who) + ": an articulated body of several bodies has no links "
                                                          "joining them (set them with am_set_constraints)");
    const long long l0 = am::g_launches.load();
    h->pairs = 0;
    cudaStream_t s = h->stream;
    am_step_stats s1{}, s2{}, uh{}, uf{};
    int rs1 = AM_OK, rs2 = AM_OK;
    // stage 1: velocities at t_k
    rc = stage_solve(h, who, t, &s1, &rs1);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->d_q0, h->d_q, 3 * h->M * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->d_th0, h->d_theta, 4 * h->M * sizeof(double), cudaMemcpyDeviceToDevice, s));
    // half step to the midpoint pose (reconstruction and correction at t_k+1/2)
    rc = set_end_links(h, dlp_half, dlq_half);
    if (rc) return rc;
    CK(cudaEventRecord(h->ev[4], s));
    rc = am::advance(h, 0.5 * dt, &uh);
    CK(cudaEventRecord(h->ev[5], s));
    if (rc) return rc;
    rc = device_flags_to_status(h, who);
    if (rc) return rc;
    if (dlpd_half) {
        CK(h2d(h->d_dlpd, dlpd_half, 3 * (size_t)h->P, s));
        CK(h2d(h->d_dlqd, dlqd_half, 3 * (size_t)h->P, s));
    }
    float ms_half = 0.f;
    CK(cudaEventSynchronize(h->ev[5]));
    cudaEventElapsedTime(&ms_half, h->ev[4], h->ev[5]);
    // stage 2: velocities at the midpoint (guess from the history, which
    // now ends with stage 1)
    rc = stage_solve(h, who, t + 0.5 * dt, &s2, &rs2);
    if (rc) return rc;
    rc = copy_outputs(h, U, phi, lam);
    if (rc) return rc;
    // full step from the pose at t_k with the midpoint velocities
    CK(cudaMemcpyAsync(h->d_q, h->d_q0, 3 * h->M * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->d_theta, h->d_th0, 4 * h->M * sizeof(double), cudaMemcpyDeviceToDevice, s));
    rc = set_end_links(h, dlp_next, dlq_next);
    if (rc) return rc;
    CK(cudaEventRecord(h->ev[4], s));
    rc = am::advance(h, dt, &uf);
    CK(cudaEventRecord(h->ev[5], s));
    CK(cudaGetLastError());
    if (rc) return rc;
    rc = device_flags_to_status(h, who);
    if (rc) return rc;
    CK(cudaStreamSynchronize(s));
    am_step_stats st{};
    st.iterations = s1.iterations + s2.iterations;
    st.restarts = s1.restarts + s2.restarts;
    st.rel_residual = std::max(s1.rel_residual, s2.rel_residual);
    st.rel_residual0 = s2.rel_residual0;
    st.constraint_residual = std::max(s1.constraint_residual, s2.constraint_residual);
    st.g2_before = uf.g2_before;
    st.g2_after = uf.g2_after;
    st.corr_iterations = std::max(uh.corr_iterations, uf.corr_iterations);
    st.ms_precond = s1.ms_precond + s2.ms_precond;
    st.ms_gmres = s1.ms_gmres + s2.ms_gmres;
    st.ms_update = ms_half + elapsed(h->ev[4], h->ev[5]);
    st.learned_systems = s1.learned_systems;
    st.pairs = h->pairs;
    st.kernel_launches = (int)(am::g_launches.load() - l0);
    const int rs = rs1 != AM_OK ? rs1 : rs2;
    st.status = rs;
    h->pc_valid = false;
    if (stats) *stats = st;
    if (rs == AM_ERR_NOT_CONVERGED) set_err(h, rs, std::string(who) + ": GMRES did not reach the tolerance");
    return rs;
}

extern "C" AM_API int am_get_bodies(am_handle* h, int system, double* q, double* theta) {
    if (!h) return AM_ERR_ARG;
    int rc = check_handle(h, "am_get_bodies", true);
    if (rc) return rc;
    rc = check_system(h, system, "am_get_bodies");
    if (rc) return rc;
    cudaStream_t s = h->stream;
    const size_t b0 = h->sys_body0[system], M = h->sys[system].M;
    if (q) CK(d2h(q, h->d_q + 3 * b0, 3 * M, s));
    if (theta) CK(d2h(theta, h->d_theta + 4 * b0, 4 * M, s));
    CK(cudaStreamSynchronize(s));
    return AM_OK;
}

extern "C" AM_API int am_get_blobs(am_handle* h, int system, double* r) {
    if (!h) return AM_ERR_ARG;
    int rc = check_handle(h, "am_get_blobs", true);
    if (rc) return rc;
    rc = check_system(h, system, "am_get_blobs");
    if (rc) return rc;
    if (!r) return set_err(h, AM_ERR_ARG, "am_get_blobs: NULL array");
    am::launch_geometry(h);
    CK(cudaGetLastError());
    am::take_flags(h);
    const size_t i0 = h->sys_blob0[system], Nb = h->sys[system].Nb;
    CK(d2h(r, h->d_r3 + 3 * i0, 3 * Nb, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return AM_OK;
}

extern "C" AM_API int am_apply_mobility(am_handle* h, const double* lam, double* u) {
    if (!h) return AM_ERR_ARG;
    int rc = check_handle(h, "am_apply_mobility", true);
    if (rc) return rc;
    if (!lam || !u) return set_err(h, AM_ERR_ARG, "am_apply_mobility: NULL array");
    cudaStream_t s = h->stream;
    am::launch_geometry(h);
    rc = device_flags_to_status(h, "am_apply_mobility");
    if (rc) return rc;
    if (h->sb) {  // (f, tau) per body in, (u, omega) per body out
        CK(h2d(h->d_t, lam, 6 * (size_t)h->M, s));
        am::sb_mobility(h, h->d_t, h->d_w);
        CK(cudaGetLastError());
        CK(d2h(u, h->d_w, 6 * (size_t)h->M, s));
        CK(cudaStreamSynchronize(s));
        return AM_OK;
    }
    if (!h->mv_tuned && am::mobility_autotune(h))
        return set_err(h, AM_ERR_CUDA, "am_apply_mobility: mobility autotuning failed");
    CK(h2d(h->d_t, lam, 3 * (size_t)h->Nb, s));
    am::mobility_apply(h, h->d_t, h->d_w, false);
    CK(cudaGetLastError());
    CK(d2h(u, h->d_w, 3 * (size_t)h->Nb, s));
    CK(cudaStreamSynchronize(s));
    return AM_OK;
}

extern "C" AM_API int am_apply_mobility_ex(am_handle* h, const double* lam, double* u, int arithmetic) {
    if (!h) return AM_ERR_ARG;
    int rc = check_handle(h, "am_apply_mobility_ex", true);
    if (rc) return rc;
    if (!lam || !u) return set_err(h, AM_ERR_ARG, "am_apply_mobility_ex: NULL array");
    int mode;
    switch (arithmetic) {
        case AM_FP64: mode = am::kOpFP64; break;
        case AM_MIXED: mode = am::kOpMixed; break;
        case AM_DF64: mode = am::kOpDF; break;
        default: return set_err(h, AM_ERR_ARG, "am_apply_mobility_ex: unknown arithmetic");
    }
    if (box_set(h->cfg)) {  // periodic: FP64 (also for double-float requests) or, on mixed handles, FP32
        if (arithmetic == AM_MIXED && h->cfg.precision != AM_MIXED)
            return set_err(h, AM_ERR_ARG, "am_apply_mobility_ex: the FP32 periodic product needs a mixed handle");
        if (arithmetic == AM_DF64) mode = am::kOpFP64;
    }
    cudaStream_t s = h->stream;
    am::launch_geometry(h);
    rc = device_flags_to_status(h, "am_apply_mobility_ex");
    if (rc) return rc;
    if (!h->mv_tuned && am::mobility_autotune(h))
        return set_err(h, AM_ERR_CUDA, "am_apply_mobility_ex: mobility autotuning failed");
    CK(h2d(h->d_t, lam, 3 * (size_t)h->Nb, s));
    am::mobility_apply(h, h->d_t, h->d_w, mode);
    CK(cudaGetLastError());
    CK(d2h(u, h->d_w, 3 * (size_t)h->Nb, s));
    CK(cudaStreamSynchronize(s));
    return AM_OK;
}

extern "C" AM_API int am_set_repulsion(am_handle* h, double eps, double range, double cutoff, double eps_wall,
                                       double range_wall) {
    if (!h) return AM_ERR_ARG;
    if (!(eps >= 0.0) || !(cutoff >= 0.0) || !(eps_wall >= 0.0) || (eps > 0.0 && !(range > 0.0)) ||
        (eps_wall > 0.0 && !(range_wall > 0.0)) || !std::isfinite(eps) || !std::isfinite(cutoff) ||
        !std::isfinite(eps_wall))
        return set_err(h, AM_ERR_ARG, "am_set_repulsion: need eps, cutoff, eps_wall >= 0 and positive ranges");
    if (eps_wall > 0.0 && !h->cfg.wall)
        return set_err(h, AM_ERR_ARG, "am_set_repulsion: wall repulsion needs a handle with a wall");
    if (eps > 0.0 && box_set(h->cfg))
        return set_err(h, AM_ERR_ARG, "am_set_repulsion: not for a periodic box");
    h->st_eps = eps;
    h->st_b = range > 0.0 ? range : 1.0;
    h->st_rc = eps > 0.0 ? cutoff : 0.0;
    h->st_eps_w = eps_wall;
    h->st_b_w = range_wall > 0.0 ? range_wall : 1.0;
    h->steric_on = (eps > 0.0 && cutoff > 0.0) || eps_wall > 0.0;
    return AM_OK;
}

extern "C" AM_API int am_steric_forces(am_handle* h, double* f) {
    if (!h) return AM_ERR_ARG;
    if (!f) return set_err(h, AM_ERR_ARG, "am_steric_forces: NULL array");
    int rc = check_handle(h, "am_steric_forces", true);
    if (rc) return rc;
    cudaStream_t s = h->stream;
    am::launch_geometry(h);
    rc = device_flags_to_status(h, "am_steric_forces");
    if (rc) return rc;
    if (h->steric_on) {
        CK(d2h(f, h->d_fst, 3 * (size_t)h->Nb, s));
    } else {
        std::fill(f, f + 3 * (size_t)h->Nb, 0.0);
    }
    CK(cudaStreamSynchronize(s));
    return AM_OK;
}

extern "C" AM_API int am_set_mobility_layout(am_handle* h, int targets_per_thread, int source_chunk) {
    if (!h) return AM_ERR_ARG;
    int rc = check_handle(h, "am_set_mobility_layout", true);
    if (rc) return rc;
    if (targets_per_thread < 0 || targets_per_thread > 3 || source_chunk < 0)
        return set_err(h, AM_ERR_ARG, "am_set_mobility_layout: targets_per_thread must be 0 .. 3 and "
                                      "source_chunk >= 0");
    if (targets_per_thread == 0) {
        h->mv_tuned = false;  // tuned again before the next product
        return AM_OK;
    }
    if (targets_per_thread == 3) {  // the symmetric product on tiles of source_chunk blobs
        const bool mixed = h->cfg.precision == AM_MIXED;
        if (box_set(h->cfg) || h->sb || (source_chunk != 32 && source_chunk != 64 && source_chunk != 128))
            return set_err(h, AM_ERR_ARG, "am_set_mobility_layout: the symmetric product needs a handle without "
                                          "a box, multi-blob bodies, and tiles of 32, 64 or 128 blobs");
        // mixed handles: paired FP32 lanes on tiles of 128, one target per lane on smaller tiles
        if (am::mobility_layout(h, mixed && source_chunk == 128 ? 2 : 1, source_chunk, 0, source_chunk / 32))
            return set_err(h, AM_ERR_CUDA, "am_set_mobility_layout: device allocation failed");
        h->mv_tuned = true;
        return AM_OK;
    }
    if (am::mobility_layout(h, targets_per_thread, source_chunk))
        return set_err(h, AM_ERR_CUDA, "am_set_mobility_layout: device allocation failed");
    h->mv_tuned = true;
    return AM_OK;
}

extern "C" AM_API int am_get_mobility_layout(am_handle* h, int* layout) {
    if (!h) return AM_ERR_ARG;
    if (!layout) return set_err(h, AM_ERR_ARG, "am_get_mobility_layout: NULL array");
    const int rc = check_handle(h, "am_get_mobility_layout", true);
    if (rc) return rc;
    layout[0] = h->mv_tpt;
    layout[1] = h->mv_chunk;
    layout[2] = h->mv_tgroup;
    layout[3] = h->n_sym > 0 ? 32 * h->sym_nsub : 0;
    return AM_OK;
}

extern "C" AM_API int am_apply_operator(am_handle* h, const double* y, double* Ay) {
    if (!h) return AM_ERR_ARG;
    int rc = check_handle(h, "am_apply_operator", true);
    if (rc) return rc;
    if (!y || !Ay) return set_err(h, AM_ERR_ARG, "am_apply_operator: NULL array");
    cudaStream_t s = h->stream;
    am::launch_geometry(h);
    rc = device_flags_to_status(h, "am_apply_operator");
    if (rc) return rc;
    if (!h->mv_tuned && am::mobility_autotune(h))
        return set_err(h, AM_ERR_CUDA, "am_apply_operator: mobility autotuning failed");
    CK(h2d(h->d_t, y, h->n, s));
    am::op_apply(h, h->d_t, h->d_w, false);
    CK(cudaGetLastError());
    CK(d2h(Ay, h->d_w, h->n, s));
    CK(cudaStreamSynchronize(s));
    return AM_OK;
}

extern "C" AM_API int am_apply_precond(am_handle* h, const double* r, double* z) {
    if (!h) return AM_ERR_ARG;
    int rc = check_handle(h, "am_apply_precond", true);
    if (rc) return rc;
    if (!r || !z) return set_err(h, AM_ERR_ARG, "am_apply_precond: NULL array");
    cudaStream_t s = h->stream;
    am::launch_geometry(h);
    am::pc_build(h);
    CK(cudaGetLastError());
    rc = device_flags_to_status(h, "am_apply_precond");
    if (rc) return rc;
    CK(h2d(h->d_t, r, h->n, s));
    am::pc_apply(h, h->d_t, h->d_z);
    CK(cudaGetLastError());
    CK(d2h(z, h->d_z, h->n, s));
    CK(cudaStreamSynchronize(s));
    return AM_OK;
}

extern "C" AM_API int am_mobility_timing(am_handle* h, int enable, double* ms, long long* launches) {
    if (!h) return AM_ERR_ARG;
    if (enable) {
        CK(cudaStreamSynchronize(h->stream));
        h->tev_used = 0;
        h->timing = true;
    } else {
        h->timing = false;
    }
    if (ms || launches) {
        CK(cudaStreamSynchronize(h->stream));
        double tot = 0.0;
        const size_t pairs = h->tev_used / 2;
        for (size_t k = 0; k < pairs; ++k) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, h->tev[2 * k], h->tev[2 * k + 1]));
            tot += t;
        }
        if (ms) *ms = tot;
        if (launches) *launches = (long long)pairs;
    }
    return AM_OK;
}

extern "C" AM_API void am_destroy(am_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_links(h);
    free_bodies(h);
    free_solver(h);
    am::periodic_free(h);
    dfree(&h->d_scal); dfree(&h->d_flags); dfree(&h->d_red); dfree(&h->d_ctrl);
    if (h->h_ctrl) cudaFreeHost(h->h_ctrl);
    for (int k = 0; k < 2; ++k) {
        if (h->gexec[k]) cudaGraphExecDestroy(h->gexec[k]);
        if (h->graph[k]) cudaGraphDestroy(h->graph[k]);
    }
    if (h->h_scal) cudaFreeHost(h->h_scal);
    if (h->h_flags) cudaFreeHost(h->h_flags);
    if (h->h_iters) cudaFreeHost(h->h_iters);
    for (int k = 0; k < 8; ++k)
        if (h->ev[k]) cudaEventDestroy(h->ev[k]);
    for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

extern "C" AM_API int am_periodic_info(am_handle* h, double* params, long long* sizes) {
    if (!h) return AM_ERR_ARG;
    if (!box_set(h->cfg)) return set_err(h, AM_ERR_ARG, "am_periodic_info: the handle has no periodic box");
    const int rc = check_handle(h, "am_periodic_info", true);
    if (rc) return rc;
    if (!h->per) return set_err(h, AM_ERR_ARG, "am_periodic_info: no bodies set");
    am::periodic_info(h, params, sizes);
    return AM_OK;
}

extern "C" AM_API const char* am_last_error(const am_handle* h) {
    if (!h) return am::thread_error();
    return h->err.c_str();
}
