// Internal declarations of libpsr shared by the mechanism loader and the kernels.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "psr.h"

namespace psr {

constexpr double kRu = 8.314462618e7;   // erg / (mol K)
constexpr double kPatm = 1.01325e6;     // dyn / cm^2, standard state of Eq. (8)
constexpr int kMaxWarpN = 64;           // K + 1 handled by one warp (two rows per lane)
// Largest batch of the persistent solvers: their int32 work-queue counter ends at B plus one
// overshooting claim per resident warp (at most 64 warps on each of at most 2^16 SMs), so
// this headroom keeps it from wrapping.
constexpr int64_t kMaxBatch = (int64_t(1) << 31) - (int64_t(1) << 22);

enum RxnType : int8_t { kElem = 0, kThirdBody = 1, kTroe = 2 };

// Per-reactor status between the two launches of a solve (never returned to the caller):
// the warp launch handed the unfinished reactor over to the block solver, which continues
// it from the iterate left in Y_out / T_out.
constexpr int32_t kStatusHandoff = 8;

// Device-side view of a mechanism: structure-of-arrays tables, all device pointers.
struct DevMech {
    int K, I, n_troe, n_eff;
    const double *W, *invW;      // [K] g/mol
    const float *invW_f;         // [K] 1/W in FP32 (the FP32 Jacobian's transform)
    const double *nasa;          // [K][16]: T_mid, low a1..a7, high a1..a7, 0
    const double *lnA, *beta, *theta;   // [I] Eq. (6), E/R in K
    const float *beta_f, *theta_f;      // [I] the same in FP32 (the FP32 Jacobian's rate derivatives)
    const int16_t *slots;        // [I][6] reactant slots 0..2, product slots 3..5, K = empty
    const int8_t *dnu;           // [I] sum_k nu_ki
    const double *dnu_d;         // [I] the same as double
    const int8_t *type;          // [I] RxnType
    const int32_t *eff_ptr;      // [I+1] CSR of (efficiency - 1) for tb/troe rows
    const int16_t *eff_sp;       // [n_eff]
    const double *eff_val;       // [n_eff] eps - 1
    const float *eff_val_f;      // [n_eff] the same in FP32
    const int32_t *troe_row;     // [I] row of troe params or -1
    const double *troe;          // [n_troe][8]: ln A0, beta0, E0/R, alpha, T3, T1, T2, 0
    const int32_t *sp_ptr;       // [K+1] CSR species -> reactions for wdot_k = sum nu_ki q_i
    const int16_t *sp_rxn;
    const int8_t *sp_nu;
    const double *sp_nu_d;       // sp_nu as double
    const int16_t *part;         // [I][6] distinct participants (K = none)
    const int8_t *part_nu;       // [I][6] net nu of each participant
    const int8_t *part_fm;       // [I][6] bit s: participant fills reactant slot s
    const int8_t *part_rm;       // [I][6] bit s: participant fills product slot s
    const int32_t *orig;         // [I] index of the reaction in the mechanism file
    int tb_first, troe_first;    // device order: elementary [0, tb_first), third-body, falloff [troe_first, I)
    int nsoot;                   // 6 when the mechanism carries MOMIC soot constants, else 0
    int soot_P, soot_H2;         // precursor and H2 species
    const double *soot;          // kSoot* layout below
};

// Soot table layout (doubles).
constexpr int kNMom = 6;
constexpr int kSootNucLnA = 0, kSootNucTheta = 1, kSootCmin = 2, kSootGrowLnA = 3, kSootGrowBeta = 4,
              kSootGrowTheta = 5, kSootGrowPref = 6, kSootKf = 7, kSootScale = 8 /* [6] s_r */,
              kSootLnScale = 14 /* [6] ln s_r */, kSootW = 20 /* [29][6] fractional-moment weights */,
              kSootWHalf = 20 + 29 * 6 /* [4] l = 1/2 weights */, kSootLen = 20 + 29 * 6 + 4;
// fractional moments: index 3 j + c for p = j + 1/6 (c = 0), j - 1/6 (c = 1), j - 1/2 (c = 2),
// j = 0..7 (coagulation); 24 + l for p = l + 2/3, l = 0..4 (growth)
constexpr int kSootNFrac = 29;

struct Mech {
    int K = 0, I = 0, E = 0, n_tb = 0, n_troe = 0, tb_first = 0, troe_first = 0;
    bool has_soot = false;
    std::vector<double> elem_w, W, comp;       // comp [K][E]
    std::vector<double> nasa;                  // [K][16]
    std::vector<double> lnA, beta, theta;
    std::vector<int16_t> slots;                // [I][6]
    std::vector<int8_t> dnu, type;
    std::vector<int32_t> eff_ptr;
    std::vector<int16_t> eff_sp;
    std::vector<double> eff_val;
    std::vector<int32_t> troe_row;
    std::vector<double> troe;
    std::vector<int32_t> sp_ptr;
    std::vector<int16_t> sp_rxn;
    std::vector<int8_t> sp_nu;
    std::vector<int16_t> part;
    std::vector<int8_t> part_nu, part_fm, part_rm;
    std::vector<int32_t> orig;
    std::vector<double> soot;                  // raw soot constants (key order of the file)
    std::vector<std::string> soot_keys;
    std::vector<double> soot_tab;              // kSootLen device table (empty without soot)
    int soot_P = 0, soot_H2 = 0;
    int device = -1;
    void *dev_block = nullptr;                 // one device allocation for all tables
    DevMech dev{};
};

int set_error(int code, const std::string &msg);
int cuda_error(const char *what, int err);

}  // namespace psr

struct psr_mech {
    psr::Mech m;
};
