// qed_step64.cu -- the plain FP64 path: one thread per particle, every operation in double precision.
// Lepton step: Sec. 5.1 (and its flow chart) with the non-emission update of Sec. 6.
// Photon step: Sec. 5.2 (and its flow chart) with the non-pair update of Sec. 6.
#include "qed_bessel.cuh"
#include "qed_internal.h"
#include "qed_steps.h"

namespace qed {

using V = V3<double>;

__device__ __forceinline__ void store_particle64(const PartDev& B, int64_t k, const V& x, const V& p, const V& s, double tau,
                                                 double w, uint64_t id) {
    B.x[k] = x.x; B.y[k] = x.y; B.z[k] = x.z;
    B.px[k] = p.x; B.py[k] = p.y; B.pz[k] = p.z;
    B.sx[k] = s.x; B.sy[k] = s.y; B.sz[k] = s.z;
    B.tau[k] = tau; B.w[k] = w; B.id[k] = id;
}

__device__ __forceinline__ bool finite3(const V& a) { return isfinite(a.x) && isfinite(a.y) && isfinite(a.z); }

enum { C_EVENTS, C_STORED, C_DROPPED, C_CLAMPED, C_RENORM, C_BELOW, C_NONFINITE, C_RATE_STEPS, C_BOUND, C_N };

__global__ void __launch_bounds__(256) lepton64_kernel(TabP<double> T, const double* __restrict__ bes, FieldP<double> F,
                                                       StepP S, double q, PartDev L, PartDev G, AppendState* A,
                                                       qed_counters* ctr) {
    const int64_t n = min(L.begin ? *L.begin : *L.count, L.capacity);
    const uint32_t fl = S.flags;
    const double dt = S.dt;
    unsigned long long c[C_N] = {};
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < n; w0 += stride) {
        const int64_t j = w0 + lane;
        bool want = false;
        V gx{0, 0, 0}, gk{0, 0, 0}, gP{0, 0, 0};
        double gtau = 0.0, gw = 0.0;
        uint64_t gid = 0;
        // the lepton's state after the step: with the event applied (st_*), and as the classical part of
        // the step left it (na_*), which it keeps if its photon finds no room
        bool st_do = false, st_event = false;
        V st_x{0, 0, 0}, st_p{0, 0, 0}, st_s{0, 0, 0}, na_p{0, 0, 0}, na_s{0, 0, 0};
        double st_tau = 0.0, na_tau = 0.0;
        if (j < n) {
            V x{L.x[j], L.y[j], L.z[j]}, p{L.px[j], L.py[j], L.pz[j]}, s{L.sx[j], L.sy[j], L.sz[j]};
            double tau = L.tau[j];
            if (!(finite3(x) && finite3(p) && finite3(s) && !isnan(tau))) {
                c[C_NONFINITE]++;
                record_error(ctr, QED_ERR_NAN, j);
            } else {
                V E, B;
                field_eval(F, S.ph_hi, 0.0, x, E, B);
                const V pold = p;
                if (fl & QED_F_PUSH) p = boris(p, E, B, q, dt);
                if (fl & QED_F_TBMT) {
                    const V pb = 0.5 * (pold + p);
                    s = rotate(s, tbmt_omega(pb, E, B, q, (fl & QED_F_TBMT_PAPER) != 0, tbmt_a(fl, T, F.eta0, pb, E, B)), dt);
                }
                const double gam = sqrt(1.0 + dot(p, p));
                if (fl & QED_F_MOVE) x = x + v3(p.x / gam * dt, p.y / gam * dt, p.z / gam * dt);
                V pf = p, sf = s;
                double tauf = tau;
                if (fl & QED_F_EMIT) {
                    const double chi = chi_of(F.eta0, gam, p, E, B);
                    const double pn = sqrt(dot(p, p));
                    V khat{0, 0, 0}, eps, beta;
                    bool ok = pn > 0.0 && chi >= S.chi_floor && chi > 0.0;
                    if (ok) {
                        khat = v3(p.x / pn, p.y / pn, p.z / pn);
                        const V v = v3(p.x / gam, p.y / gam, p.z / gam);
                        ok = make_basis(E, B, v, khat, -q, eps, beta);
                    }
                    if (ok) {
                        const double lnchi = log(chi);
                        if (chi > T.chi_max) c[C_CLAMPED]++;
                        double Iu, Id;
                        nlc_rates(T, chi, lnchi, Iu, Id);
                        const double pref = kAlpha / (kSqrt3 * kPi * F.eta0 * gam);
                        const double Wu = pref * Iu, Wd = pref * Id;
                        const bool resolved = (fl & QED_F_RESOLVED) != 0;
                        const double sb = resolved ? dot(s, beta) : 0.0;
                        const double Wup = Wu * (1.0 + sb) / 2.0, Wdn = Wd * (1.0 - sb) / 2.0;
                        const double Ws = Wup + Wdn;
                        bool event = false, down = false;
                        double u0a = 0.0, rej_up = 0.0;
                        const uint64_t id = L.id[j];
                        if (fl & QED_F_REJECT) {
                            // table-free (Sec. 4.2): candidate lambda = r1^3, accepted with probability
                            // 3 r1^2 (dW/dlambda) dt, dW/dlambda = pref w(lambda; s.beta) (App. A.1)
                            const uint4 w = draw(id, S.seed, S.step, kSlotTauBranch);
                            const double r1 = uniform52(w.x, w.y), r2 = uniform52(w.z, w.w);
                            const double lc = r1 * r1 * r1, om = 1.0 - lc;
                            rej_up = 2.0 * lc / (3.0 * chi * om);
                            double b[3] = {0.0, 0.0, 0.0};
                            if (rej_up < 700.0) bessel64(bes, rej_up, b);  // scaled by e^{u'}; beyond, w ~ 0
                            const double wl = (-b[2] + (1.0 / om + om) * b[1] + lc * sb * b[0]) * exp(-rej_up);
                            const double acc = 3.0 * r1 * r1 * pref * wl * dt;
                            if (acc > 1.0) c[C_BOUND]++;
                            event = r2 < acc;
                        } else if (fl & QED_F_TAU) {
                            tauf = tau - Ws * dt;
                            event = tauf <= 0.0;
                            if (event) {
                                const uint4 w = draw(id, S.seed, S.step, kSlotTauBranch);
                                u0a = uniform52(w.x, w.y);
                                down = uniform52(w.z, w.w) * Ws < Wdn;
                            }
                        } else {
                            const uint4 w = draw(id, S.seed, S.step, kSlotTauBranch);
                            u0a = uniform52(w.x, w.y);
                            event = u0a < Ws * dt;
                            down = u0a < Wdn * dt;
                        }
                        if (event) {
                            st_event = true;
                            na_p = p;
                            na_s = s;
                            na_tau = tauf;  // spent (optical depth) or unchanged (probability mode)
                            const uint4 w1 = draw(id, S.seed, S.step, kSlotLambdaSpin);
                            const uint4 w2 = draw(id, S.seed, S.step, kSlotStokes);
                            const double r2 = uniform52(w1.x, w1.y), r3 = uniform52(w1.z, w1.w), r4 = uniform52(w2.x, w2.y);
                            const double y = log(r2) - log(1.0 - r2);
                            const double up = (fl & QED_F_REJECT) ? rej_up : exp(icdf_lookup(T, false, down ? 1 : 0, lnchi, y));
                            const double lam = 3.0 * chi * up / (2.0 + 3.0 * chi * up);
                            const double one_m = 1.0 - lam;
                            const V k = lam * p;
                            if (fl & QED_F_RECOIL) pf = one_m * p;
                            double b[3];
                            bessel64(bes, up, b);
                            V si{0, 0, 0}, sfu{0, 0, 0};
                            if (resolved) si = s;
                            double xi[3] = {0.0, 0.0, 0.0};
                            double wv = 0.0;
                            V g{0, 0, 0};
                            if (fl & (QED_F_SPIN_EVENT | QED_F_POL_EVENT)) nlc_wg(lam, one_m, b, si, beta, khat, wv, g);
                            if (fl & QED_F_SPIN_EVENT) {
                                const double gn = sqrt(dot(g, g));
                                if (fl & QED_F_BETA_BASIS) {  // resolved along +-beta (Sec. 8.3 comparison)
                                    const double gb = dot(g, beta);
                                    sf = (fl & QED_F_SPIN_COLLAPSE) ? (r3 < (wv - gb) / (2.0 * wv) ? -1.0 : 1.0) * beta
                                                                    : (gb / wv) * beta;
                                } else if (fl & QED_F_SPIN_COLLAPSE) {
                                    const double sg = r3 < (wv - gn) / (2.0 * wv) ? -1.0 : 1.0;
                                    sf = gn > 0.0 ? v3(sg * g.x / gn, sg * g.y / gn, sg * g.z / gn) : v3(0.0, 0.0, 0.0);
                                } else {
                                    sf = v3(g.x / wv, g.y / wv, g.z / wv);
                                }
                                sfu = sf;
                            }
                            if (fl & QED_F_POL_EVENT) {
                                double Fv[4];
                                nlc_stokes(lam, one_m, b, si, sfu, wv, g, eps, beta, khat, Fv);
                                const double Fn = sqrt(Fv[1] * Fv[1] + Fv[2] * Fv[2] + Fv[3] * Fv[3]);
                                if (fl & QED_F_POL_COLLAPSE) {
                                    const double sg = r4 < (Fv[0] - Fn) / (2.0 * Fv[0]) ? -1.0 : 1.0;
                                    for (int i = 0; i < 3; ++i) xi[i] = Fn > 0.0 ? sg * Fv[i + 1] / Fn : 0.0;
                                } else {
                                    for (int i = 0; i < 3; ++i) xi[i] = Fv[i + 1] / Fv[0];
                                }
                            }
                            if ((fl & QED_F_TAU) && !(fl & QED_F_REJECT)) tauf = -log(u0a);
                            const uint4 wc = draw(id, S.seed, S.step, kSlotChild);
                            const double kn = sqrt(dot(k, k));
                            if (kn >= S.store_min) {
                                want = true;
                                gx = x;
                                gk = k;
                                gP = stokes_to_P(xi, eps, beta, khat);
                                gid = (uint64_t)wc.x | ((uint64_t)wc.y << 32);
                                gtau = birth_tau(gid, S.seed);
                                gw = L.w[j];
                            } else {
                                c[C_BELOW]++;
                            }
                        } else if ((fl & QED_F_NONTRANSITION) && resolved) {
                            const double W0 = 0.5 * (Wu + Wd), Pi = 0.5 * (Wu - Wd);
                            const double D = 1.0 - (W0 + Pi * dot(beta, s)) * dt;
                            if (D > 0.0) {
                                sf = v3((s.x * (1.0 - W0 * dt) - Pi * beta.x * dt) / D, (s.y * (1.0 - W0 * dt) - Pi * beta.y * dt) / D,
                                        (s.z * (1.0 - W0 * dt) - Pi * beta.z * dt) / D);
                                const double n2 = dot(sf, sf);
                                if (n2 > 1.0) {
                                    const double nn = sqrt(n2);
                                    sf = v3(sf.x / nn, sf.y / nn, sf.z / nn);
                                    c[C_RENORM]++;
                                }
                            }
                        }
                        // the loop's Scorer term (App. A.1): a turn about the rest-frame magnetic field
                        if (!event && (fl & QED_F_LOOP)) sf = rotate(sf, loop_omega(T, F.eta0, chi, gam, p, E, B, q), dt);
                    }
                }
                st_do = true;
                st_x = x;
                st_p = pf;
                st_s = sf;
                st_tau = tauf;
            }
        }
        // the photon's slot: event ev of the call writes base + ev if ev < budget; otherwise the event
        // is not applied (the lepton keeps its pre-event state and its spent optical depth)
        const long long ev = reserve_event(A, want);
        const bool keep = want && A != nullptr && ev < A->budget;
        const bool refused = want && A != nullptr && !keep;
        if (keep) {
            store_particle64(G, A->base[0] + ev, gx, gk, gP, gtau, gw, gid);
            c[C_STORED]++;
        }
        if (refused) {
            c[C_DROPPED]++;
            record_error(ctr, QED_ERR_CAPACITY, j);
        } else if (want && A == nullptr) {
            c[C_DROPPED]++;  // the caller keeps no photons
        }
        if (st_event && !refused) c[C_EVENTS]++;
        if (st_do) {
            const V op = refused ? na_p : st_p, os = refused ? na_s : st_s;
            L.x[j] = st_x.x; L.y[j] = st_x.y; L.z[j] = st_x.z;
            L.px[j] = op.x; L.py[j] = op.y; L.pz[j] = op.z;
            L.sx[j] = os.x; L.sy[j] = os.y; L.sz[j] = os.z;
            L.tau[j] = refused ? na_tau : st_tau;
        }
    }
    flush_counters<C_N>(c, &ctr->events);
}

__global__ void __launch_bounds__(256) photon64_kernel(TabP<double> T, const double* __restrict__ bes, FieldP<double> F,
                                                       StepP S, PartDev G, PartDev El, PartDev Po, AppendState* A,
                                                       qed_counters* ctr) {
    const int64_t n = min(G.begin ? *G.begin : *G.count, G.capacity);
    const uint32_t fl = S.flags;
    const double dt = S.dt;
    unsigned long long c[C_N] = {};
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool have_daughters = El.count != nullptr && Po.count != nullptr;
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < n; w0 += stride) {
        const int64_t j = w0 + lane;
        bool want = false;
        V x{0, 0, 0}, k{0, 0, 0}, Pf{0, 0, 0}, pe{0, 0, 0}, pp{0, 0, 0}, se{0, 0, 0}, sp{0, 0, 0};
        double tauf = 0.0, te = 0.0, tp = 0.0, wgt = 0.0;
        uint64_t ide = 0, idp = 0;
        bool skip = true;
        if (j < n) {
            x = v3(G.x[j], G.y[j], G.z[j]);
            k = v3(G.px[j], G.py[j], G.pz[j]);
            const V P{G.sx[j], G.sy[j], G.sz[j]};
            const double tau = G.tau[j];
            if (!(finite3(x) && finite3(k) && finite3(P) && !isnan(tau))) {
                c[C_NONFINITE]++;
                record_error(ctr, QED_ERR_NAN, j);
            } else {
                skip = false;
                V E, B;
                field_eval(F, S.ph_hi, 0.0, x, E, B);
                const double en = sqrt(dot(k, k));
                V khat{0, 0, 0};
                if (en > 0.0) khat = v3(k.x / en, k.y / en, k.z / en);
                if (fl & QED_F_MOVE) x = x + dt * khat;
                Pf = P;
                tauf = tau;
                if ((fl & QED_F_EMIT) && en > 0.0) {
                    const double chi = chi_of(F.eta0, en, k, E, B);
                    V eps, beta;
                    const bool ok = chi >= S.chi_floor && chi > 0.0 && make_basis(E, B, khat, khat, 1.0, eps, beta);
                    if (ok) {
                        const bool resolved = (fl & QED_F_RESOLVED) != 0;
                        double xi[3];
                        P_to_stokes(P, eps, beta, khat, xi);
                        if (!resolved) xi[0] = xi[1] = xi[2] = 0.0;
                        const double lnchi = log(chi);
                        if (chi > T.chi_max) c[C_CLAMPED]++;
                        double Jp, Jm;
                        nbw_rates(T, chi, lnchi, Jp, Jm);
                        const double pref = kAlpha / (kSqrt3 * kPi * F.eta0 * en);
                        const double Wp = pref * Jp, Wm = pref * Jm;
                        const double Wmp = Wm * (1.0 - xi[2]) / 2.0, Wpp = Wp * (1.0 + xi[2]) / 2.0;
                        const double Wx = Wmp + Wpp;
                        bool event = false, minus = false;
                        double rej_lam = 0.0, rej_ut = 0.0;
                        const uint64_t id = G.id[j];
                        if (fl & QED_F_REJECT) {
                            // table-free (Sec. 4.2): candidate positron fraction lambda = r1, accepted with
                            // probability (dW/dlambda) dt = pref w0(lambda; xi3) dt (App. A.2)
                            const uint4 w = draw(id, S.seed, S.step, kSlotTauBranch);
                            const double r1 = uniform52(w.x, w.y), r2 = uniform52(w.z, w.w);
                            const double om = 1.0 - r1;
                            rej_lam = r1;
                            rej_ut = 2.0 / (3.0 * chi * r1 * om);
                            double b[3] = {0.0, 0.0, 0.0};
                            if (rej_ut < 700.0) bessel64(bes, rej_ut, b);  // scaled by e^{u~'}; beyond, w0 ~ 0
                            const double w0r = (b[2] + (om / r1 + r1 / om) * b[1] - xi[2] * b[1]) * exp(-rej_ut);
                            const double acc = pref * w0r * dt;
                            if (acc > 1.0) c[C_BOUND]++;
                            event = r2 < acc;
                        } else if (fl & QED_F_TAU) {
                            tauf = tau - Wx * dt;
                            event = tauf <= 0.0;
                            if (event) {
                                const uint4 w = draw(id, S.seed, S.step, kSlotTauBranch);
                                minus = uniform52(w.z, w.w) * Wx < Wmp;
                            }
                        } else {
                            const uint4 w = draw(id, S.seed, S.step, kSlotTauBranch);
                            const double r1 = uniform52(w.x, w.y);
                            event = r1 < Wx * dt;
                            minus = r1 < Wmp * dt;
                        }
                        if (event && ((fl & QED_F_REJECT) || Wx > 0.0)) {
                            const uint4 w1 = draw(id, S.seed, S.step, kSlotLambdaSpin);
                            const double r = uniform52(w1.x, w1.y), r3 = uniform52(w1.z, w1.w);
                            double ut, lam;
                            if (fl & QED_F_REJECT) {
                                ut = rej_ut;
                                lam = rej_lam;
                            } else {
                                const double rf = r < 0.5 ? 1.0 - 2.0 * r : 2.0 * r - 1.0;
                                double xv = 0.0;
                                if (rf > 0.0) xv = exp(icdf_lookup(T, true, minus ? 1 : 0, lnchi, log(rf) - log(1.0 - rf)));
                                ut = 8.0 / (3.0 * chi) + xv;
                                const double qq = 2.0 / (3.0 * chi * ut);
                                const double mu = 0.5 * (1.0 - sqrt(1.0 - 4.0 * qq));
                                lam = r < 0.5 ? mu : 1.0 - mu;
                            }
                            const double one_m = 1.0 - lam;
                            double b[3];
                            bessel64(bes, ut, b);
                            pp = lam * k;
                            pe = one_m * k;
                            if (fl & QED_F_SPIN_EVENT) {
                                double w0v;
                                V je, jp;
                                nbw_j(lam, one_m, b, xi, eps, beta, khat, w0v, je, jp);
                                if (fl & QED_F_SPIN_COLLAPSE) {
                                    const double jen = sqrt(dot(je, je)), jpn = sqrt(dot(jp, jp));
                                    V Se = jen > 0.0 ? v3(je.x / jen, je.y / jen, je.z / jen) : v3(0.0, 0.0, 0.0);
                                    V Sp = jpn > 0.0 ? v3(jp.x / jpn, jp.y / jpn, jp.z / jpn) : v3(0.0, 0.0, 0.0);
                                    if (fl & QED_F_BETA_BASIS) Se = Sp = beta;  // the G_ab sum to 4 w0 on any axes
                                    // four correlated states, order (--, -+, +-, ++), first sign = positron
                                    double cum = 0.0;
                                    int chosen = 3;
                                    for (int a = 0; a < 4; ++a) {
                                        const double sa = (a & 2) ? 1.0 : -1.0, sbb = (a & 1) ? 1.0 : -1.0;
                                        cum += nbw_G(lam, one_m, b, xi, sa * Sp, sbb * Se, eps, beta, khat) / (4.0 * w0v);
                                        if (r3 < cum) {
                                            chosen = a;
                                            break;
                                        }
                                    }
                                    const double sa = (chosen & 2) ? 1.0 : -1.0, sbb = (chosen & 1) ? 1.0 : -1.0;
                                    sp = sa * Sp;
                                    se = sbb * Se;
                                } else if (fl & QED_F_BETA_BASIS) {
                                    se = (dot(je, beta) / w0v) * beta;
                                    sp = (dot(jp, beta) / w0v) * beta;
                                } else {
                                    se = v3(je.x / w0v, je.y / w0v, je.z / w0v);
                                    sp = v3(jp.x / w0v, jp.y / w0v, jp.z / w0v);
                                }
                            }
                            const uint4 wc = draw(id, S.seed, S.step, kSlotChild);
                            ide = (uint64_t)wc.x | ((uint64_t)wc.y << 32);
                            idp = (uint64_t)wc.z | ((uint64_t)wc.w << 32);
                            te = birth_tau(ide, S.seed);
                            tp = birth_tau(idp, S.seed);
                            wgt = G.w[j];
                            want = true;
                        } else if (!event && (fl & QED_F_NONTRANSITION) && resolved) {
                            const double W0 = 0.5 * (Wp + Wm), Pi = 0.5 * (Wp - Wm);
                            const double D = 1.0 - (W0 + Pi * xi[2]) * dt;
                            if (D > 0.0) {
                                double xn[3] = {xi[0] * (1.0 - W0 * dt) / D, xi[1] * (1.0 - W0 * dt) / D,
                                                (xi[2] * (1.0 - W0 * dt) - Pi * dt) / D};
                                const double n2 = xn[0] * xn[0] + xn[1] * xn[1] + xn[2] * xn[2];
                                if (n2 > 1.0) {
                                    const double nn = sqrt(n2);
                                    for (int i = 0; i < 3; ++i) xn[i] /= nn;
                                    c[C_RENORM]++;
                                }
                                Pf = stokes_to_P(xn, eps, beta, khat);
                            }
                        }
                    }
                }
            }
        }
        // daughters: one reservation for the pair (electron base[0] + ev, positron base[1] + ev), both or
        // neither
        bool ok = false;
        if (have_daughters) {
            const long long ev = reserve_event(A, want);
            ok = want && ev < A->budget;
            if (ok) {
                store_particle64(El, A->base[0] + ev, x, pe, se, te, wgt, ide);
                store_particle64(Po, A->base[1] + ev, x, pp, sp, tp, wgt, idp);
            }
            const long long s_d = reserve_slots(G.n_dead, ok, 1);
            if (ok && s_d < G.capacity) G.dead[s_d] = j;
        }
        if (want) {
            if (ok) {
                c[C_EVENTS]++;
                c[C_STORED] += 2;
            } else {
                c[C_DROPPED]++;
                if (have_daughters) record_error(ctr, QED_ERR_CAPACITY, j);
            }
        }
        if (j < n && !skip) {
            G.x[j] = x.x; G.y[j] = x.y; G.z[j] = x.z;
            if (ok) {  // converted: inert until compaction
                G.px[j] = 0.0; G.py[j] = 0.0; G.pz[j] = 0.0;
                G.w[j] = 0.0;
            } else {
                G.sx[j] = Pf.x; G.sy[j] = Pf.y; G.sz[j] = Pf.z;
            }
            G.tau[j] = tauf;
        }
    }
    flush_counters<C_N>(c, &ctr->events);
}

}  // namespace qed

void launch_lepton64(const qed_tables_s* t, const qed_field& f, const qed_step_desc& s, const qed_particles* L,
                     const qed_particles* G, qed_counters* ctr, cudaStream_t st) {
    using namespace qed;
    StepP S = step_params(s, f);
    PartDev g{};
    if (G) g = part_dev(G);
    const int blocks = launch_blocks(L->capacity, 256);
    lepton64_kernel<<<blocks, 256, 0, st>>>(tab_params<double>(t), t->bes64, field_params<double>(f), S, (double)L->charge,
                                            part_dev(L), g, G ? append_state(ctr) : nullptr, ctr);
}

void launch_photon64(const qed_tables_s* t, const qed_field& f, const qed_step_desc& s, const qed_particles* G,
                     const qed_particles* El, const qed_particles* Po, qed_counters* ctr, cudaStream_t st) {
    using namespace qed;
    StepP S = step_params(s, f);
    PartDev e{}, p{};
    if (El && Po) {
        e = part_dev(El);
        p = part_dev(Po);
    }
    const int blocks = launch_blocks(G->capacity, 256);
    photon64_kernel<<<blocks, 256, 0, st>>>(tab_params<double>(t), t->bes64, field_params<double>(f), S, part_dev(G), e, p,
                                            (El && Po) ? append_state(ctr) : nullptr, ctr);
}
