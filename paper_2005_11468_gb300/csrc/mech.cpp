// Mechanism loader: parses `.psrmech` text, derives the tables the kernels read and
// uploads them to the current device in one allocation.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>

#include "psr_internal.h"

namespace psr {

static thread_local std::string g_err;

int set_error(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_error(const char *what, int err) {
    return set_error(PSR_E_CUDA, std::string(what) + ": " +
                                     cudaGetErrorString(static_cast<cudaError_t>(err)));
}

namespace {

struct Lines {
    std::vector<std::vector<std::string>> rows;
    size_t pos = 0;
    bool next(std::vector<std::string> &r) {
        if (pos >= rows.size()) return false;
        r = rows[pos++];
        return true;
    }
};

bool to_d(const std::string &s, double &v) {
    char *end = nullptr;
    v = std::strtod(s.c_str(), &end);
    return end && *end == '\0' && std::isfinite(v);
}
bool to_i(const std::string &s, long &v) {
    char *end = nullptr;
    v = std::strtol(s.c_str(), &end, 10);
    return end && *end == '\0';
}

// Lagrange weights l_j(p) of the polynomial through nodes 0..nn-1.
void lagrange(int nn, double p, double *w) {
    for (int j = 0; j < nn; ++j) {
        double v = 1.0;
        for (int k = 0; k < nn; ++k)
            if (k != j) v *= (p - k) / double(j - k);
        w[j] = v;
    }
}

// MOMIC constants: nucleation, growth prefactor chi_alpha pi d_C^2, coagulation
// K_f / sqrt(T), moment scales, and the interpolation weights of every fractional
// moment the sources use (p >= 0: nodes 0..5; p < 0: quadratic over 0, 1, 2).
int build_soot(Mech &m) {
    auto get = [&](const char *key, double &v) {
        for (size_t j = 0; j < m.soot_keys.size(); ++j)
            if (m.soot_keys[j] == key) {
                v = m.soot[j];
                return true;
            }
        return false;
    };
    double P, H2, nA, nth, cmin, gA, gb, gth, chi, rho_s, eps, m0f;
    if (!get("precursor", P) || !get("h2", H2) || !get("nuc_A", nA) || !get("nuc_theta", nth) ||
        !get("cmin", cmin) || !get("grow_A", gA) || !get("grow_beta", gb) || !get("grow_theta", gth) ||
        !get("chi_alpha", chi) || !get("rho_s", rho_s) || !get("coag_eps", eps) || !get("m0_floor", m0f))
        return set_error(PSR_E_FORMAT, "psrmech: soot record lacks a constant");
    if (P < 0 || P >= m.K || H2 < 0 || H2 >= m.K || !(nA > 0) || !(cmin >= 1) || gA < 0 || !(chi >= 0) ||
        !(rho_s > 0) || eps < 0 || !(m0f > 0))
        return set_error(PSR_E_FORMAT, "psrmech: soot constant out of range");
    constexpr double kNA = 6.02214076e23, kKB = 1.380649e-16, kPi = 3.14159265358979323846;
    const double mC = 12.011 / kNA;
    const double dC = std::cbrt(6.0 * mC / (kPi * rho_s));
    std::vector<double> t(kSootLen, 0.0);
    t[kSootNucLnA] = std::log(nA);
    t[kSootNucTheta] = nth;
    t[kSootCmin] = cmin;
    t[kSootGrowLnA] = gA > 0 ? std::log(gA) : -1e300;
    t[kSootGrowBeta] = gb;
    t[kSootGrowTheta] = gth;
    t[kSootGrowPref] = chi * kPi * dC * dC;
    t[kSootKf] = eps * std::pow(3.0 * mC / (4.0 * kPi * rho_s), 1.0 / 6.0) * std::sqrt(6.0 * kKB / rho_s);
    for (int r = 0; r < kNMom; ++r) {
        t[kSootScale + r] = m0f * std::pow(cmin, r);
        t[kSootLnScale + r] = std::log(t[kSootScale + r]);
    }
    for (int idx = 0; idx < kSootNFrac; ++idx) {
        double p;
        if (idx < 24) {
            const int j = idx / 3, c = idx % 3;
            p = j + (c == 0 ? 1.0 / 6.0 : (c == 1 ? -1.0 / 6.0 : -0.5));
        } else {
            p = (idx - 24) + 2.0 / 3.0;
        }
        double *w = t.data() + kSootW + idx * kNMom;
        if (p >= 0) lagrange(kNMom, p, w);
        else lagrange(3, p, w);
    }
    lagrange(4, 0.5, t.data() + kSootWHalf);
    m.soot_tab = t;
    m.soot_P = static_cast<int>(P);
    m.soot_H2 = static_cast<int>(H2);
    return PSR_OK;
}

int parse(const std::string &text, Mech &m) {
    Lines L;
    std::istringstream in(text);
    std::string line;
    while (std::getline(in, line)) {
        std::istringstream ls(line);
        std::vector<std::string> toks;
        std::string t;
        while (ls >> t) toks.push_back(t);
        if (toks.empty() || toks[0][0] == '#') continue;
        L.rows.push_back(toks);
    }
    std::vector<std::string> r;
    auto bad = [&](const std::string &what) {
        return set_error(PSR_E_FORMAT, "psrmech: " + what);
    };
    if (!L.next(r) || r.size() < 2 || r[0] != "psrmech" || r[1] != "1") return bad("missing 'psrmech 1' header");
    long E = 0, K = 0, I = 0, v = 0;
    if (!L.next(r) || r.size() != 2 || r[0] != "elements" || !to_i(r[1], E) || E < 1 || E > 16)
        return bad("bad 'elements' record");
    m.E = static_cast<int>(E);
    for (long e = 0; e < E; ++e) {
        double w;
        if (!L.next(r) || r.size() != 2 || !to_d(r[1], w) || w <= 0) return bad("bad element record");
        m.elem_w.push_back(w);
    }
    if (!L.next(r) || r.size() != 2 || r[0] != "species" || !to_i(r[1], K) || K < 1 || K > 30000)
        return bad("bad 'species' record");
    m.K = static_cast<int>(K);
    m.comp.assign(K * E, 0.0);
    m.nasa.assign(K * 16, 0.0);
    m.W.assign(K, 0.0);
    for (long k = 0; k < K; ++k) {
        if (!L.next(r) || (long)r.size() != 2 + E + 3 + 14 || !to_i(r[0], v) || v != k)
            return bad("bad species record " + std::to_string(k));
        double w = 0;
        for (long e = 0; e < E; ++e) {
            double a;
            if (!to_d(r[2 + e], a) || a < 0) return bad("bad composition of species " + std::to_string(k));
            m.comp[k * E + e] = a;
            w += a * m.elem_w[e];
        }
        if (w <= 0) return bad("species " + std::to_string(k) + " has no atoms");
        m.W[k] = w;
        double vals[17];
        for (int j = 0; j < 17; ++j)
            if (!to_d(r[2 + E + j], vals[j])) return bad("bad thermo of species " + std::to_string(k));
        m.nasa[k * 16 + 0] = vals[1];                   // T_mid
        for (int j = 0; j < 7; ++j) m.nasa[k * 16 + 1 + j] = vals[3 + j];    // low range
        for (int j = 0; j < 7; ++j) m.nasa[k * 16 + 8 + j] = vals[10 + j];   // high range
    }
    if (!L.next(r) || r.size() != 2 || r[0] != "reactions" || !to_i(r[1], I) || I < 1 || I > 32767)
        return bad("bad 'reactions' record");
    m.I = static_cast<int>(I);
    m.slots.assign(I * 6, static_cast<int16_t>(K));
    m.dnu.assign(I, 0);
    m.type.assign(I, kElem);
    m.lnA.assign(I, 0.0);
    m.beta.assign(I, 0.0);
    m.theta.assign(I, 0.0);
    m.troe_row.assign(I, -1);
    m.eff_ptr.assign(I + 1, 0);
    std::vector<std::vector<std::pair<int, double>>> effs(I);
    std::vector<std::array<double, 8>> troe_par(I);
    for (long i = 0; i < I; ++i) {
        if (!L.next(r) || r.size() < 4 || !to_i(r[0], v) || v != i)
            return bad("bad reaction record " + std::to_string(i));
        const std::string &kind = r[1];
        if (kind == "elem") m.type[i] = kElem;
        else if (kind == "tb") m.type[i] = kThirdBody;
        else if (kind == "troe") m.type[i] = kTroe;
        else return bad("unknown reaction type '" + kind + "'");
        size_t p = 2;
        int dn = 0;
        for (int side = 0; side < 2; ++side) {
            long n;
            if (p >= r.size() || !to_i(r[p], n) || n < 1 || n > 3)
                return bad("reaction " + std::to_string(i) + ": 1..3 species per side");
            ++p;
            for (long s = 0; s < n; ++s) {
                long sp;
                if (p >= r.size() || !to_i(r[p], sp) || sp < 0 || sp >= K)
                    return bad("reaction " + std::to_string(i) + ": bad species index");
                m.slots[i * 6 + side * 3 + s] = static_cast<int16_t>(sp);
                dn += side ? 1 : -1;
                ++p;
            }
        }
        m.dnu[i] = static_cast<int8_t>(dn);
        double A, b, th;
        if (p + 3 > r.size() || !to_d(r[p], A) || !to_d(r[p + 1], b) || !to_d(r[p + 2], th) || A <= 0)
            return bad("reaction " + std::to_string(i) + ": bad Arrhenius parameters");
        m.lnA[i] = std::log(A);
        m.beta[i] = b;
        m.theta[i] = th;
        p += 3;
        double low[3] = {0, 0, 0}, troe[4] = {0, 0, 0, 0};
        bool has_low = false, has_troe = false;
        while (p < r.size()) {
            if (r[p] == "low" && p + 3 < r.size()) {
                for (int j = 0; j < 3; ++j)
                    if (!to_d(r[p + 1 + j], low[j])) return bad("reaction " + std::to_string(i) + ": bad low");
                if (low[0] <= 0) return bad("reaction " + std::to_string(i) + ": A0 <= 0");
                has_low = true;
                p += 4;
            } else if (r[p] == "troe" && p + 4 < r.size()) {
                for (int j = 0; j < 4; ++j)
                    if (!to_d(r[p + 1 + j], troe[j])) return bad("reaction " + std::to_string(i) + ": bad troe");
                has_troe = true;
                p += 5;
            } else if (r[p] == "eff" && p + 1 < r.size()) {
                long ne;
                if (!to_i(r[p + 1], ne) || ne < 0 || ne > K) return bad("reaction " + std::to_string(i) + ": bad eff");
                p += 2;
                for (long e = 0; e < ne; ++e) {
                    long sp;
                    double ev;
                    if (p + 1 >= r.size() || !to_i(r[p], sp) || sp < 0 || sp >= K || !to_d(r[p + 1], ev) || ev < 0)
                        return bad("reaction " + std::to_string(i) + ": bad efficiency");
                    effs[i].push_back({static_cast<int>(sp), ev - 1.0});
                    p += 2;
                }
            } else {
                return bad("reaction " + std::to_string(i) + ": unknown field '" + r[p] + "'");
            }
        }
        if (m.type[i] == kTroe) {
            if (!has_low || !has_troe) return bad("falloff reaction " + std::to_string(i) + " needs low and troe");
            if (troe[1] <= 0 || troe[2] <= 0) return bad("falloff reaction " + std::to_string(i) + ": T3, T1 > 0");
            troe_par[i] = {std::log(low[0]), low[1], low[2], troe[0], troe[1], troe[2], troe[3], 0.0};
            m.n_troe++;
        } else if (has_low || has_troe) {
            return bad("reaction " + std::to_string(i) + ": low/troe on a non-falloff reaction");
        }
        if (m.type[i] == kThirdBody) m.n_tb++;
        if (m.type[i] == kElem && !effs[i].empty()) return bad("reaction " + std::to_string(i) + ": eff on elementary");
    }
    while (L.next(r)) {
        if (r[0] == "soot") {
            m.has_soot = true;
            for (size_t j = 1; j + 1 < r.size(); j += 2) {
                double x;
                if (!to_d(r[j + 1], x)) return bad("bad soot constant '" + r[j] + "'");
                m.soot_keys.push_back(r[j]);
                m.soot.push_back(x);
            }
        } else if (r[0] == "end") {
            break;
        } else {
            return bad("unexpected record '" + r[0] + "'");
        }
    }
    // Device order of the reactions: elementary, then third-body, then falloff, so that
    // warps sweeping the reaction list meet one rate form per pass; orig maps back to
    // the file's index (used for per-reaction inputs such as rate multipliers).
    std::vector<int32_t> ord;
    for (int want : {int(kElem), int(kThirdBody), int(kTroe)})
        for (long i = 0; i < I; ++i)
            if (m.type[i] == want) ord.push_back(static_cast<int32_t>(i));
    {
        auto perm = [&](auto &v, int width) {
            auto old = v;
            for (long i = 0; i < I; ++i)
                for (int c = 0; c < width; ++c) v[i * width + c] = old[size_t(ord[i]) * width + c];
        };
        perm(m.lnA, 1);
        perm(m.beta, 1);
        perm(m.theta, 1);
        perm(m.slots, 6);
        perm(m.dnu, 1);
        perm(m.type, 1);
        auto e_old = effs;
        auto t_old = troe_par;
        for (long i = 0; i < I; ++i) {
            effs[i] = e_old[ord[i]];
            troe_par[i] = t_old[ord[i]];
        }
        m.orig = ord;
    }
    m.troe_first = static_cast<int>(I) - m.n_troe;
    m.tb_first = m.troe_first - m.n_tb;
    for (long i = m.troe_first; i < I; ++i) {
        m.troe_row[i] = static_cast<int32_t>(i - m.troe_first);
        m.troe.insert(m.troe.end(), troe_par[i].begin(), troe_par[i].end());
    }
    // efficiency CSR
    for (long i = 0; i < I; ++i) {
        m.eff_ptr[i + 1] = m.eff_ptr[i] + static_cast<int32_t>(effs[i].size());
        for (auto &e : effs[i]) {
            m.eff_sp.push_back(static_cast<int16_t>(e.first));
            m.eff_val.push_back(e.second);
        }
    }
    // distinct participants, net stoichiometry and the slots each occupies;
    // species -> reaction CSR (Eq. (4))
    m.part.assign(I * 6, static_cast<int16_t>(K));
    m.part_nu.assign(I * 6, 0);
    m.part_fm.assign(I * 6, 0);
    m.part_rm.assign(I * 6, 0);
    std::vector<std::vector<std::pair<int, int>>> by_sp(K);
    for (long i = 0; i < I; ++i) {
        std::map<int, int> nu;
        std::map<int, int> fm, rm;
        for (int s = 0; s < 6; ++s) {
            int sp = m.slots[i * 6 + s];
            if (sp < K) {
                nu[sp] += (s < 3) ? -1 : 1;
                if (s < 3) fm[sp] |= 1 << s;
                else rm[sp] |= 1 << (s - 3);
            }
        }
        int j = 0;
        for (auto &kv : nu) {
            m.part[i * 6 + j] = static_cast<int16_t>(kv.first);
            m.part_nu[i * 6 + j] = static_cast<int8_t>(kv.second);
            m.part_fm[i * 6 + j] = static_cast<int8_t>(fm[kv.first]);
            m.part_rm[i * 6 + j] = static_cast<int8_t>(rm[kv.first]);
            ++j;
            if (kv.second != 0) by_sp[kv.first].push_back({static_cast<int>(i), kv.second});
        }
    }
    if (m.has_soot) {
        int rc = build_soot(m);
        if (rc != PSR_OK) return rc;
    }
    m.sp_ptr.assign(K + 1, 0);
    for (long k = 0; k < K; ++k) {
        m.sp_ptr[k + 1] = m.sp_ptr[k] + static_cast<int32_t>(by_sp[k].size());
        for (auto &e : by_sp[k]) {
            m.sp_rxn.push_back(static_cast<int16_t>(e.first));
            m.sp_nu.push_back(static_cast<int8_t>(e.second));
        }
    }
    return PSR_OK;
}

template <class T>
void place(std::vector<char> &blob, const std::vector<T> &v, size_t &off_out) {
    size_t off = (blob.size() + 255) & ~size_t(255);
    blob.resize(off + v.size() * sizeof(T) + 1);
    if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
    off_out = off;
}

int upload(Mech &m) {
    std::vector<char> blob;
    std::vector<double> invW(m.K);
    for (int k = 0; k < m.K; ++k) invW[k] = 1.0 / m.W[k];
    std::vector<float> invW_f(invW.begin(), invW.end()), eff_val_f(m.eff_val.begin(), m.eff_val.end());
    std::vector<float> beta_f(m.beta.begin(), m.beta.end()), theta_f(m.theta.begin(), m.theta.end());
    size_t oinvWf, oeffvf, obetaf, othetaf;
    size_t oW, oinvW, onasa, olnA, obeta, otheta, oslots, odnu, otype, oeffp, oeffs, oeffv, otr, otroe,
        osp, ospr, ospn, opart, opartnu, opfm, oprm, oorig, odnud, ospnd, osoot;
    std::vector<double> dnu_d(m.dnu.begin(), m.dnu.end()), sp_nu_d(m.sp_nu.begin(), m.sp_nu.end());
    place(blob, m.W, oW);
    place(blob, invW, oinvW);
    place(blob, invW_f, oinvWf);
    place(blob, eff_val_f, oeffvf);
    place(blob, beta_f, obetaf);
    place(blob, theta_f, othetaf);
    place(blob, m.nasa, onasa);
    place(blob, m.lnA, olnA);
    place(blob, m.beta, obeta);
    place(blob, m.theta, otheta);
    place(blob, m.slots, oslots);
    place(blob, m.dnu, odnu);
    place(blob, m.type, otype);
    place(blob, m.eff_ptr, oeffp);
    place(blob, m.eff_sp, oeffs);
    place(blob, m.eff_val, oeffv);
    place(blob, m.troe_row, otr);
    place(blob, m.troe, otroe);
    place(blob, m.sp_ptr, osp);
    place(blob, m.sp_rxn, ospr);
    place(blob, m.sp_nu, ospn);
    place(blob, m.part, opart);
    place(blob, m.part_nu, opartnu);
    place(blob, m.part_fm, opfm);
    place(blob, m.part_rm, oprm);
    place(blob, m.orig, oorig);
    place(blob, dnu_d, odnud);
    place(blob, sp_nu_d, ospnd);
    place(blob, m.soot_tab, osoot);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error("cudaGetDevice", e);
    void *d = nullptr;
    e = cudaMalloc(&d, blob.size());
    if (e != cudaSuccess) return set_error(PSR_E_OOM, "cudaMalloc of mechanism tables failed");
    e = cudaMemcpy(d, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_error("cudaMemcpy mechanism", e);
    }
    char *b = static_cast<char *>(d);
    m.device = dev;
    m.dev_block = d;
    DevMech &D = m.dev;
    D.K = m.K;
    D.I = m.I;
    D.n_troe = m.n_troe;
    D.n_eff = static_cast<int>(m.eff_sp.size());
    D.W = reinterpret_cast<const double *>(b + oW);
    D.invW = reinterpret_cast<const double *>(b + oinvW);
    D.invW_f = reinterpret_cast<const float *>(b + oinvWf);
    D.eff_val_f = reinterpret_cast<const float *>(b + oeffvf);
    D.beta_f = reinterpret_cast<const float *>(b + obetaf);
    D.theta_f = reinterpret_cast<const float *>(b + othetaf);
    D.nasa = reinterpret_cast<const double *>(b + onasa);
    D.lnA = reinterpret_cast<const double *>(b + olnA);
    D.beta = reinterpret_cast<const double *>(b + obeta);
    D.theta = reinterpret_cast<const double *>(b + otheta);
    D.slots = reinterpret_cast<const int16_t *>(b + oslots);
    D.dnu = reinterpret_cast<const int8_t *>(b + odnu);
    D.type = reinterpret_cast<const int8_t *>(b + otype);
    D.eff_ptr = reinterpret_cast<const int32_t *>(b + oeffp);
    D.eff_sp = reinterpret_cast<const int16_t *>(b + oeffs);
    D.eff_val = reinterpret_cast<const double *>(b + oeffv);
    D.troe_row = reinterpret_cast<const int32_t *>(b + otr);
    D.troe = reinterpret_cast<const double *>(b + otroe);
    D.sp_ptr = reinterpret_cast<const int32_t *>(b + osp);
    D.sp_rxn = reinterpret_cast<const int16_t *>(b + ospr);
    D.sp_nu = reinterpret_cast<const int8_t *>(b + ospn);
    D.part = reinterpret_cast<const int16_t *>(b + opart);
    D.part_nu = reinterpret_cast<const int8_t *>(b + opartnu);
    D.part_fm = reinterpret_cast<const int8_t *>(b + opfm);
    D.part_rm = reinterpret_cast<const int8_t *>(b + oprm);
    D.orig = reinterpret_cast<const int32_t *>(b + oorig);
    D.dnu_d = reinterpret_cast<const double *>(b + odnud);
    D.sp_nu_d = reinterpret_cast<const double *>(b + ospnd);
    D.nsoot = m.has_soot ? kNMom : 0;
    D.soot_P = m.soot_P;
    D.soot_H2 = m.soot_H2;
    D.soot = m.has_soot ? reinterpret_cast<const double *>(b + osoot) : nullptr;
    D.tb_first = m.tb_first;
    D.troe_first = m.troe_first;
    return PSR_OK;
}

int load_text(const std::string &text, psr_mech **out) {
    if (!out) return set_error(PSR_E_ARG, "psr_mech_load: out is NULL");
    *out = nullptr;
    auto *pm = new (std::nothrow) psr_mech();
    if (!pm) return set_error(PSR_E_OOM, "host allocation failed");
    int rc = parse(text, pm->m);
    if (rc == PSR_OK) rc = upload(pm->m);
    if (rc != PSR_OK) {
        delete pm;
        return rc;
    }
    *out = pm;
    return PSR_OK;
}

}  // namespace
}  // namespace psr

extern "C" {

int psr_mech_load(const char *path, psr_mech **out) {
    if (!path) return psr::set_error(PSR_E_ARG, "psr_mech_load: path is NULL");
    std::ifstream f(path, std::ios::binary);
    if (!f) return psr::set_error(PSR_E_IO, std::string("cannot open ") + path);
    std::stringstream ss;
    ss << f.rdbuf();
    return psr::load_text(ss.str(), out);
}

int psr_mech_load_mem(const char *text, size_t nbytes, psr_mech **out) {
    if (!text) return psr::set_error(PSR_E_ARG, "psr_mech_load_mem: text is NULL");
    return psr::load_text(std::string(text, nbytes), out);
}

int psr_mech_info_get(const psr_mech *m, psr_mech_info *out) {
    if (!m || !out) return psr::set_error(PSR_E_ARG, "psr_mech_info_get: NULL argument");
    out->K = m->m.K;
    out->I = m->m.I;
    out->n_elements = m->m.E;
    out->n_third_body = m->m.n_tb;
    out->n_falloff = m->m.n_troe;
    out->has_soot = m->m.has_soot ? 1 : 0;
    return PSR_OK;
}

int psr_mech_weights(const psr_mech *m, double *W_out) {
    if (!m || !W_out) return psr::set_error(PSR_E_ARG, "psr_mech_weights: NULL argument");
    std::memcpy(W_out, m->m.W.data(), sizeof(double) * m->m.K);
    return PSR_OK;
}

void psr_mech_free(psr_mech *m) {
    if (!m) return;
    if (m->m.dev_block) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != m->m.device && m->m.device >= 0) cudaSetDevice(m->m.device);
        cudaFree(m->m.dev_block);
        if (cur >= 0 && cur != m->m.device) cudaSetDevice(cur);
    }
    delete m;
}

const char *psr_last_error(void) { return psr::g_err.c_str(); }

void psr_options_default(psr_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->ftol = 1e-8;
    o->step_rtol = 1e-10;
    o->step_atol_y = 1e-14;
    o->step_atol_t = 1e-10;
    o->ts_rtol = 1e-4;
    o->ts_atol_y = 1e-10;
    o->dt0_over_tau = 1e-6;
    o->dt_shrink = 0.25;
    o->y_floor = 1e-10;
    o->t_min = 200.0;
    o->t_max = 5000.0;
    o->max_newton = 500;
    o->max_damp = 8;
    o->max_ts_rounds = 100;
    o->ts_steps = 12;
    o->ts_newton = 8;
    o->precision = PSR_FP64;
    o->energy = PSR_ADIABATIC;
    o->mixed_fallback = 2;
    o->jacobian = PSR_JAC_ANALYTIC;
    o->mixed_max_newton = -1;
    o->jac_age = 1;
    o->ts_linear = 150;
    o->handoff = -1;
}

}  // extern "C"
