// Host-side circuit records and fusion plans.
#pragma once

#include <string>
#include <vector>

#include "internal.h"

namespace qsim {

struct GateRec {
    int kind = 0;
    int k = 0;
    int nc = 0;
    int targets[QSIM_MAX_TARGETS] = {};
    int controls[QSIM_MAX_CONTROLS] = {};
    double params[4] = {};
    int pindex = -1;
    int grad_slot = -1;  // adjoint reverse sweeps only: gradient marker on targets[0]
    double grad_v[3] = {0, 0, 0};  // its operator px X + py Y + pz Z
    std::vector<cd> m;  // the gate's matrix (2^k x 2^k), built at insertion
};

// A fused gate: matrix on an ordered qubit list (qubits[0] = MSB of its index).
struct Block {
    std::vector<int> qubits;
    std::vector<cd> m;
    std::vector<int> gates;  // indices of the source gates, in order
};

// Device-side copies of a block plan for one precision.
struct PlanDev {
    bool ready = false;
    std::vector<Op> ops;
    std::vector<size_t> mat_off;
    void *mats = nullptr;
};

struct StagedPlan;  // staged.cu
struct TcPlan;      // tc.cu

std::vector<cd> embed_gate(const GateRec &g, const std::vector<int> &qs);
std::vector<cd> matmul(const std::vector<cd> &A, const std::vector<cd> &B, size_t D);
std::vector<cd> widen(const std::vector<cd> &m, const std::vector<int> &from, const std::vector<int> &to);

}  // namespace qsim

struct qsim_circuit {
    int n = 0;
    std::vector<qsim::GateRec> gates;
    int nparams = 0;
};

struct qsim_plan {
    int n = 0;
    int mode = 0;
    int kmax = 2;
    int ngates = 0;
    double tuned_ms = -1.0;  // autotuned plans: time per run measured by the autotuner
    std::vector<qsim::Block> blocks;  // GREEDY2 and TC block lists
    qsim::PlanDev dev[2];
    qsim::StagedPlan *staged = nullptr;
    qsim::TcPlan *tc = nullptr;
    int nsweeps() const;
    void release_staged();
    void release_tc();
    ~qsim_plan();
};

namespace qsim {
int build_greedy2(const qsim_circuit &c, qsim_plan &p);
int build_staged(const qsim_circuit &c, qsim_plan &p);
int run_staged(qsim_state *s, qsim_plan &p);
// staged plans whose tile stages run as kernels compiled for the plan
void staged_set_specialized(qsim_plan &p);
bool staged_specialized(const qsim_plan &p);
constexpr int SPECIALIZE_MIN_QUBITS = 20;  // the autotuner's specialised candidates
int staged_nsweeps(const qsim_plan &p);
void staged_describe(const qsim_plan &p, std::string &out);
void tc_describe(const qsim_plan &p, std::string &out);
int build_tc(const qsim_circuit &c, qsim_plan &p);
int run_tc(qsim_state *s, qsim_plan &p);
int tc_nsweeps(const qsim_plan &p);
int tc_set_precisions(qsim_plan &p, const std::vector<int> &prec);
int tc_pass_precision(const qsim_plan &p, int i);
int run_block_plan(qsim_state *s, qsim_plan &p);
}  // namespace qsim
