// Host-side FP64 set-up of the mixed basis: knots, B-spline tables on the
// Gauss planes, banded S and D with the Cholesky factor of S, cutoff discs,
// the local pseudopotential's terms grouped by profile (the table on the
// quadrature planes is built from them on the device) and the
// Kleinman-Bylander factors.  Runs once per handle; nothing here is on the
// apply path.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <tuple>

#include "mb_internal.h"

namespace mb {

namespace {

const double kPi = 3.14159265358979323846;

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's iteration on P_n,
// evaluated with the three-term recurrence (Golub & Welsch give the same rule
// as eigenvalues; Newton from Tricomi's initial guess is the classic route).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int m = 2; m <= n; ++m) {
                double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? z : p1;
            double pm = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute derivative at the converged node
        double p0 = 1.0, p1 = z;
        for (int m = 2; m <= n; ++m) {
            double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
            p0 = p1;
            p1 = p2;
        }
        double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
        dp = n * (z * pn - pm) / (z * z - 1.0);
        x[n - 1 - i] = z;   // ascending
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// The `ord` B-splines of order `ord` that are non-zero on [tau[l], tau[l+1]),
// B_{l-ord+1 .. l}(z), by the triangular form of the recursion Eq. (1)
// (de Boor's BSPLVB arrangement: left/right knot distances, one pass per order).
void nonzero_bsplines(const std::vector<double> &tau, int l, int ord, double z, double *b) {
    double dl[16], dr[16];
    b[0] = 1.0;
    for (int j = 1; j < ord; ++j) {
        dr[j] = tau[l + j] - z;
        dl[j] = z - tau[l + 1 - j];
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            double den = dr[r + 1] + dl[j - r];
            double term = den != 0.0 ? b[r] / den : 0.0;
            b[r] = saved + dr[r + 1] * term;
            saved = dl[j - r] * term;
        }
        b[j] = saved;
    }
}

}  // namespace

int build_host_tables(mb_handle *h, const mb_cell *cell, const double *kpts, int nk,
                      double ecut, const double *breaks, int nbreaks, int order,
                      const mb_atom *atoms, int natoms, const mb_opts *opts) {
    if (!cell || !kpts || nk <= 0 || !breaks || nbreaks < 2 || !opts) return MB_EINVAL;
    if (order < 3 || order > 8) return MB_EINVAL;
    if (!(ecut > 0.0)) return MB_EINVAL;
    if (natoms < 0 || (natoms > 0 && !atoms)) return MB_EINVAL;
    for (int i = 1; i < nbreaks; ++i)
        if (!(breaks[i] > breaks[i - 1])) return MB_EINVAL;
    int nint = nbreaks - 1;
    if (nint < order) return MB_EINVAL;
    auto pow2 = [](int v, int &lg) {
        if (v < 4 || v > 256) return false;
        lg = 0;
        while ((1 << lg) < v) ++lg;
        return (1 << lg) == v;
    };
    if (!pow2(opts->n1, h->l1) || !pow2(opts->n2, h->l2)) return MB_EINVAL;
    h->n1 = opts->n1;
    h->n2 = opts->n2;
    h->order = order;
    h->nquad = opts->nquad > 0 ? opts->nquad : order;
    if (h->nquad > 16) return MB_EINVAL;
    h->nint = nint;
    h->nb = nint + order - 3;
    h->nq = nint * h->nquad;
    h->ecut = ecut;
    h->max_bands = opts->max_bands > 0 ? opts->max_bands : 128;
    h->precond_shift = opts->precond_shift > 0 ? opts->precond_shift : 1.0;
    for (int i = 0; i < 2; ++i) {
        h->a1[i] = cell->a1[i];
        h->a2[i] = cell->a2[i];
    }
    double det = h->a1[0] * h->a2[1] - h->a1[1] * h->a2[0];
    if (!(std::fabs(det) > 1e-12)) return MB_EINVAL;
    h->Ac = std::fabs(det);
    // b_i . a_j = 2 pi delta_ij
    h->b1[0] = 2 * kPi * h->a2[1] / det;
    h->b1[1] = -2 * kPi * h->a2[0] / det;
    h->b2[0] = -2 * kPi * h->a1[1] / det;
    h->b2[1] = 2 * kPi * h->a1[0] / det;

    // ---- knots and Gauss planes
    h->breaks.assign(breaks, breaks + nbreaks);
    h->tau.clear();
    for (int i = 0; i < order - 1; ++i) h->tau.push_back(breaks[0]);
    for (int i = 0; i < nbreaks; ++i) h->tau.push_back(breaks[i]);
    for (int i = 0; i < order - 1; ++i) h->tau.push_back(breaks[nbreaks - 1]);
    std::vector<double> gx, gw;
    gauss_legendre(h->nquad, gx, gw);
    const int K = order, P = h->nquad, nq = h->nq, nb = h->nb;
    h->zq.resize(nq);
    h->wq.resize(nq);
    h->Bq.assign((size_t)nq * K, 0.0);
    std::vector<double> dBq((size_t)nq * K, 0.0);
    for (int t = 0; t < nint; ++t) {
        double lo = breaks[t], hi = breaks[t + 1], hh = hi - lo;
        int l = K - 1 + t;
        for (int s = 0; s < P; ++s) {
            int q = t * P + s;
            double z = lo + 0.5 * hh * (gx[s] + 1.0);
            h->zq[q] = z;
            h->wq[q] = 0.5 * hh * gw[s];
            double b[16], bl[16];
            nonzero_bsplines(h->tau, l, K, z, b);        // B_{t .. t+K-1}
            nonzero_bsplines(h->tau, l, K - 1, z, bl);   // order K-1: B_{t+1 .. t+K-1}
            for (int m = 0; m < K; ++m) {
                h->Bq[(size_t)q * K + m] = b[m];
                // Eq. (3): B'_{i,K} = (K-1)[B_{i,K-1}/(tau_{i+K-1}-tau_i) - B_{i+1,K-1}/(tau_{i+K}-tau_{i+1})]
                int i = t + m;
                double lower_i = (m >= 1) ? bl[m - 1] : 0.0;      // B_{i,K-1}
                double lower_i1 = (m <= K - 2) ? bl[m] : 0.0;     // B_{i+1,K-1}
                double d1 = h->tau[i + K - 1] - h->tau[i];
                double d2 = h->tau[i + K] - h->tau[i + 1];
                double v = 0.0;
                if (d1 > 0) v += lower_i / d1;
                if (d2 > 0) v -= lower_i1 / d2;
                dBq[(size_t)q * K + m] = (K - 1) * v;
            }
        }
    }

    // ---- banded S, D over retained splines j = full index - 1
    const int W = 2 * K - 1;
    h->Sb.assign((size_t)nb * W, 0.0);
    h->Db.assign((size_t)nb * W, 0.0);
    for (int q = 0; q < nq; ++q) {
        int t = q / P;
        for (int m = 0; m < K; ++m) {
            int j = t + m - 1;
            if (j < 0 || j >= nb) continue;
            for (int m2 = 0; m2 < K; ++m2) {
                int j2 = t + m2 - 1;
                if (j2 < 0 || j2 >= nb) continue;
                int d = j2 - j + (K - 1);
                h->Sb[(size_t)j * W + d] += h->wq[q] * h->Bq[(size_t)q * K + m] * h->Bq[(size_t)q * K + m2];
                h->Db[(size_t)j * W + d] += h->wq[q] * dBq[(size_t)q * K + m] * dBq[(size_t)q * K + m2];
            }
        }
    }
    // banded Cholesky S = L L^T, L[j][j-d] stored at Lb[j*K + d]
    h->Lb.assign((size_t)nb * K, 0.0);
    for (int j = 0; j < nb; ++j) {
        for (int d = K - 1; d >= 0; --d) {
            int i = j - d;                       // column
            if (i < 0) continue;
            double s = h->Sb[(size_t)i * W + (j - i) + (K - 1)];   // S[i][j]
            for (int c = std::max(0, j - (K - 1)); c < i; ++c)
                s -= h->Lb[(size_t)j * K + (j - c)] * h->Lb[(size_t)i * K + (i - c)];
            if (d == 0) {
                if (!(s > 0.0)) return MB_EINVAL;
                h->Lb[(size_t)j * K] = std::sqrt(s);
            } else {
                h->Lb[(size_t)j * K + d] = s / h->Lb[(size_t)i * K];
            }
        }
    }

    // ---- cutoff discs
    h->kp.assign(nk, KPoint());
    h->kofs.assign(nk + 1, 0);
    h->qofs.assign(nk + 1, 0);
    double r = std::sqrt(2.0 * ecut);
    double la1 = std::hypot(h->a1[0], h->a1[1]), la2 = std::hypot(h->a2[0], h->a2[1]);
    for (int ik = 0; ik < nk; ++ik) {
        KPoint &kp = h->kp[ik];
        kp.k[0] = kpts[2 * ik];
        kp.k[1] = kpts[2 * ik + 1];
        double kn = std::hypot(kp.k[0], kp.k[1]);
        int lim1 = (int)std::ceil((r + kn) * la1 / (2 * kPi)) + 1;
        int lim2 = (int)std::ceil((r + kn) * la2 / (2 * kPi)) + 1;
        std::vector<std::tuple<int, int, int>> gl;   // (goff, n1, n2)
        for (int a = -lim1; a <= lim1; ++a)
            for (int b = -lim2; b <= lim2; ++b) {
                double qx = kp.k[0] + a * h->b1[0] + b * h->b2[0];
                double qy = kp.k[1] + a * h->b1[1] + b * h->b2[1];
                if (0.5 * (qx * qx + qy * qy) <= ecut) {
                    if (2 * std::abs(a) + 1 > h->n1 || 2 * std::abs(b) + 1 > h->n2) return MB_EINVAL;
                    int i1 = ((a % h->n1) + h->n1) % h->n1, i2 = ((b % h->n2) + h->n2) % h->n2;
                    gl.emplace_back(i1 * h->n2 + i2, a, b);
                }
            }
        if (gl.empty()) return MB_EINVAL;
        // disc order: by n2, then n1 -- column by column of the grid, so that
        // consecutive G of a warp sit one compact-plane row apart (a stride
        // of N2 + 1 elements, free of shared-memory bank conflicts)
        std::sort(gl.begin(), gl.end(), [](const std::tuple<int, int, int> &x, const std::tuple<int, int, int> &y) {
            return std::make_pair(std::get<2>(x), std::get<1>(x)) < std::make_pair(std::get<2>(y), std::get<1>(y));
        });
        kp.ng = (int)gl.size();
        kp.ldg = (kp.ng + 31) / 32 * 32;
        for (auto &e : gl) {
            kp.goff.push_back(std::get<0>(e));
            int a = std::get<1>(e), b = std::get<2>(e);
            kp.n1.push_back(a);
            kp.n2.push_back(b);
            double qx = kp.k[0] + a * h->b1[0] + b * h->b2[0];
            double qy = kp.k[1] + a * h->b1[1] + b * h->b2[1];
            kp.qx.push_back(qx);
            kp.qy.push_back(qy);
            kp.q2.push_back(qx * qx + qy * qy);
        }
        h->kofs[ik + 1] = h->kofs[ik] + kp.ldg;
    }
    h->total_ldg = h->kofs[nk];

    // ---- local pseudopotential (Eq. (10)): the terms, grouped by profile
    // (kind, width, height); the table V(r, z_q) is built from them on the
    // device when the handle's tables are uploaded
    {
        std::map<std::tuple<int, double, double>, std::vector<std::array<double, 3>>> groups;
        for (int i = 0; i < natoms; ++i) {
            const mb_atom &at = atoms[i];
            if (at.A != 0.0) {
                if (!(at.w > 0.0)) return MB_EINVAL;
                groups[{0, 1.0 / (2.0 * at.w * at.w), at.pos[2]}].push_back({at.A, at.pos[0], at.pos[1]});
            }
            if (at.Z != 0.0) {
                if (!(at.Rcore > 0.0) || !std::isfinite(at.Z)) return MB_EINVAL;
                groups[{1, at.Rcore, at.pos[2]}].push_back({at.Z, at.pos[0], at.pos[1]});
            }
        }
        h->lgrp.clear();
        h->lion.clear();
        h->lstart.assign(1, 0);
        for (auto &gr : groups) {
            h->lgrp.insert(h->lgrp.end(), {(double)std::get<0>(gr.first), std::get<1>(gr.first), std::get<2>(gr.first)});
            for (auto &ion : gr.second) h->lion.insert(h->lion.end(), ion.begin(), ion.end());
            h->lstart.push_back((int)(h->lion.size() / 3));
        }
        if (groups.empty()) h->lstart.clear();
    }

    // ---- Kleinman-Bylander projectors (Eqs. (14)-(17)) as separable terms
    // zproj[t][j] * qproj[t][G].  Per atom: 1s, p_x, p_y, p_z (one term each)
    // and, with nproj = 5, 2s = C2 (Z_{1,00} Q_{2,00} + Z_{2,00} Q_{1,00}).
    h->nterm = 0;
    h->nkb = 0;
    for (int i = 0; i < natoms; ++i) {
        if (atoms[i].nproj != 0 && atoms[i].nproj != 4 && atoms[i].nproj != 5) return MB_EINVAL;
        if (atoms[i].nproj > 0 && !(atoms[i].rc > 0)) return MB_EINVAL;
        h->nkb += atoms[i].nproj;
        h->nterm += atoms[i].nproj == 5 ? 6 : atoms[i].nproj;
    }
    const int NP = h->nterm;
    h->zproj.assign((size_t)NP * nb, 0.0);
    h->Ekb.assign(h->nkb, 0.0);
    h->Ecoup.assign(h->nkb, 0.0);
    h->Qkb.assign(h->nkb, 0.0);
    h->Qcoup.assign(h->nkb, 0.0);
    h->aug.clear();
    h->partner.assign(h->nkb, -1);
    h->tproj.assign(NP, 0);
    h->pstart.assign(h->nkb + 1, 0);
    h->plist.clear();
    for (int ik = 0; ik < nk; ++ik) {
        h->kp[ik].qproj.assign((size_t)NP * h->kp[ik].ldg, cdouble(0.0));
        h->qofs[ik + 1] = h->qofs[ik] + NP * h->kp[ik].ldg;
    }
    int tt = 0, pp = 0;
    for (int i = 0; i < natoms; ++i) {
        if (atoms[i].nproj == 0) continue;
        const mb_atom &at = atoms[i];
        const bool two_s = at.nproj == 5;
        double al = 1.0 / (2.0 * at.rc * at.rc);
        double Cs = std::pow(2.0 * al / kPi, 0.75);
        double Cp = 2.0 * std::sqrt(al) * Cs;
        // int (r^2)^2 exp(-2 alpha r^2) d^3r = 4 pi (15/16) sqrt(pi) (2 alpha)^(-7/2)
        double C2 = 1.0 / std::sqrt(4.0 * kPi * 15.0 / 16.0 * std::sqrt(kPi) * std::pow(2.0 * al, -3.5));
        // terms of this atom: 0 1s, 1 p_x, 2 p_y, 3 p_z, [4 2s: Z_{1,00} Q_{2,00}, 5 2s: Z_{2,00} Q_{1,00}]
        const int nt = two_s ? 6 : 4;
        const int zkind[6] = {0, 0, 0, 1, 0, 2};   // Z_{1,00}, Z_{1,10}, Z_{2,00}
        for (int q = 0; q < nq; ++q) {
            int t = q / P;
            double dz = h->zq[q] - at.pos[2];
            double g = h->wq[q] * std::exp(-al * dz * dz);
            const double zf[3] = {g, g * dz, g * dz * dz};
            for (int m = 0; m < K; ++m) {
                int j = t + m - 1;
                if (j < 0 || j >= nb) continue;
                double bv = h->Bq[(size_t)q * K + m];
                for (int c = 0; c < nt; ++c) h->zproj[(size_t)(tt + c) * nb + j] += zf[zkind[c]] * bv;
            }
        }
        for (int c = 0; c < 4; ++c) h->Ekb[pp + c] = at.E[c];
        for (int c = 0; c < 4; ++c) h->Qkb[pp + c] = at.q[c];
        for (int c = 0; c < nt; ++c) h->tproj[tt + c] = pp + (c < 4 ? c : 4);
        if (two_s) {
            h->Ekb[pp + 4] = at.E2s;
            h->partner[pp] = pp + 4;
            h->partner[pp + 4] = pp;
            h->Ecoup[pp] = h->Ecoup[pp + 4] = at.E12;
            h->Qkb[pp + 4] = at.q2s;
            h->Qcoup[pp] = h->Qcoup[pp + 4] = at.q12;
        }
        bool aug = false;
        for (int c = 0; c < at.nproj; ++c) aug = aug || h->Qkb[pp + c] != 0.0 || h->Qcoup[pp + c] != 0.0;
        if (aug) {
            if (!(at.rQ > 0.0)) return MB_EINVAL;
            h->aug.push_back({pp, at.nproj, at.pos[0], at.pos[1], at.pos[2], at.rQ});
        }
        for (int ik = 0; ik < nk; ++ik) {
            KPoint &kp = h->kp[ik];
            for (int g = 0; g < kp.ng; ++g) {
                double qx = kp.qx[g], qy = kp.qy[g];
                double Qs = (kPi / al) * std::exp(-kp.q2[g] / (4 * al));
                double Q2 = (1.0 / al - kp.q2[g] / (4 * al * al)) * Qs;   // Q_{2,00}
                cdouble ph = std::polar(1.0 / std::sqrt(h->Ac), -(qx * at.pos[0] + qy * at.pos[1]));
                // conj of C*Q: Q_x = i q_x/(2 alpha) Q_s  ->  conj = -i q_x/(2 alpha) Q_s
                kp.qproj[(size_t)(tt + 0) * kp.ldg + g] = ph * (Cs * Qs);
                kp.qproj[(size_t)(tt + 1) * kp.ldg + g] = ph * cdouble(0.0, -Cp * qx / (2 * al) * Qs);
                kp.qproj[(size_t)(tt + 2) * kp.ldg + g] = ph * cdouble(0.0, -Cp * qy / (2 * al) * Qs);
                kp.qproj[(size_t)(tt + 3) * kp.ldg + g] = ph * (Cp * Qs);
                if (two_s) {
                    kp.qproj[(size_t)(tt + 4) * kp.ldg + g] = ph * (C2 * Q2);
                    kp.qproj[(size_t)(tt + 5) * kp.ldg + g] = ph * (C2 * Qs);
                }
            }
        }
        tt += nt;
        pp += at.nproj;
    }
    h->uspp = !h->aug.empty();
    for (int p = 0; p < h->nkb; ++p) {
        for (int t = 0; t < NP; ++t)
            if (h->tproj[t] == p) h->plist.push_back(t);
        h->pstart[p + 1] = (int)h->plist.size();
    }
    // group terms by identical z factor (s, p_x, p_y and the first 2s term of
    // an atom share one; atoms at one height with one radius share theirs)
    h->nzf = 0;
    h->zfun.clear();
    h->pgroup.assign(NP, -1);
    h->zstart.assign(1, 0);
    h->zlist.clear();
    for (int p0 = 0; p0 < NP; ++p0) {
        if (h->pgroup[p0] >= 0) continue;
        const double *r0 = h->zproj.data() + (size_t)p0 * nb;
        const int f = h->nzf++;
        h->zfun.insert(h->zfun.end(), r0, r0 + nb);
        for (int p1 = p0; p1 < NP; ++p1) {
            const double *r1 = h->zproj.data() + (size_t)p1 * nb;
            if (h->pgroup[p1] < 0 && std::equal(r0, r0 + nb, r1)) {
                h->pgroup[p1] = f;
                h->zlist.push_back(p1);
            }
        }
        h->zstart.push_back((int)h->zlist.size());
    }
    return MB_OK;
}

// Banded Cholesky factors of T(G) + c S = D/2 + (|k+G|^2/2 + c) S for every
// G of k-point ik, stored G-fastest: out[(j*K + d)*ldg + g] = L_G[j][j-d]
// for d >= 1 and 1 / L_G[j][j] for d = 0.
void precond_factors(const mb_handle *h, int ik, double shift, std::vector<double> &out) {
    const int K = h->order, W = 2 * K - 1, nb = h->nb;
    const KPoint &kp = h->kp[ik];
    const size_t ldg = kp.ldg;
    out.assign(ldg * nb * K, 0.0);
    std::vector<double> L((size_t)nb * K);
    for (int g = 0; g < kp.ldg; ++g) {
        std::fill(L.begin(), L.end(), 0.0);
        double qq = g < kp.ng ? 0.5 * kp.q2[g] + shift : shift;
        for (int j = 0; j < nb; ++j) {
            for (int d = K - 1; d >= 0; --d) {
                int i = j - d;
                if (i < 0) continue;
                size_t idx = (size_t)i * W + (j - i) + (K - 1);
                double s = 0.5 * h->Db[idx] + qq * h->Sb[idx];
                for (int c = std::max(0, j - (K - 1)); c < i; ++c)
                    s -= L[(size_t)j * K + (j - c)] * L[(size_t)i * K + (i - c)];
                if (d == 0)
                    L[(size_t)j * K] = std::sqrt(s > 0 ? s : 1e-300);
                else
                    L[(size_t)j * K + d] = s / L[(size_t)i * K];
            }
        }
        // stored with the reciprocal of the diagonal (the solves multiply by it)
        for (int j = 0; j < nb; ++j)
            for (int d = 0; d < K; ++d)
                out[((size_t)j * K + d) * ldg + g] = d == 0 ? 1.0 / L[(size_t)j * K] : L[(size_t)j * K + d];
    }
}

}  // namespace mb
