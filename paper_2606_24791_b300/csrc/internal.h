// Internal declarations of the B300 LAMG+ library (not part of the public ABI).
#pragma once

#include <cstdint>
#include <string>
#include <functional>
#include <vector>

#include <cuda_runtime.h>

#include "lamg.h"

namespace lamg {

enum LevelKind { KIND_ELIM = 0, KIND_AGG = 1, KIND_COARSEST = 2 };

// Level operator on the host: off-diagonal CSR (columns ascending) + diagonal.
struct HostMat {
    int64_t n = 0;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> val;
    std::vector<double> diag;
    int64_t nnz() const { return (int64_t)ci.size(); }
};

// One level of the hierarchy in the caller's (natural) numbering.
struct HostLevel {
    int kind = KIND_COARSEST;
    HostMat A;
    std::vector<int32_t> colour;  // aggregation levels
    int ncol = 0;
    int64_t nc = 0;               // coarse size (elimination: |C|, aggregation: aggregates)
    std::vector<int32_t> cidx;    // elimination: coarse index or -1
    std::vector<int32_t> agg, agg2;
    std::vector<double> wt;
    std::vector<double> X;        // test vectors n x K (lamg_setup only)
    std::vector<double> aff;      // per off-diagonal entry (lamg_setup only)
    std::vector<uint8_t> strong;  // per off-diagonal entry (lamg_setup only)
    std::vector<uint8_t> adm;     // strong and passes the energy-ratio guard (lamg_setup only)
    std::vector<double> pinv;     // coarsest: dense pseudo-inverse
    double gamma = 0.0;
    // Chebyshev smoothing instead of Gauss-Seidel (aggregation levels with many colours):
    // step k of one polynomial is d <- c1[k] d + c2[k] D^{-1}(b - A x), x <- x + d
    int cheb = 0;
    double cheb_lambda = 0.0, cheb_c1[8] = {0}, cheb_c2[8] = {0};
};

struct Status {
    int code = LAMG_OK;
    std::string msg;
};

// Host threads one setup may use: min(16, hardware threads). (Measured: giving each of the
// server's concurrent setups an equal share of the host made served latency worse; a setup's
// own latency is what a request waits for.)
int setup_threads();

// host setup (setup_host.cpp)
int validate_graph(const lamg_graph *g);
// Setup phases timed by build_hierarchy and finalize (milliseconds, lamg_setup_times).
enum SetupPhase {
    SETUP_INPUT = 0,     // validation and Laplacian
    SETUP_ELIM,          // degree-<=4 independent set and Schur complement (Eq. 2)
    SETUP_COLOUR,        // greedy colouring
    SETUP_TV_AFFINITY,   // test vectors and affinities on the GPU, with their copies
    SETUP_AGGREGATE,     // guarded aggregation and caliber-2 (Eqs. 3-4, 9, 13)
    SETUP_GALERKIN,      // P^T A P
    SETUP_DENSE,         // dense pseudo-inverse of the coarsest level
    SETUP_DEVICE,        // device orders, uploads, sliced copies
    SETUP_SCHEDULE,      // step list, kernel-form timing, cluster choice, graph capture
    SETUP_NPHASE
};
int build_hierarchy(const lamg_graph *g, const lamg_options &o, std::vector<HostLevel> &levels,
                    double *times = nullptr);
int greedy_colour(const HostMat &A, std::vector<int32_t> &colour);
// Chebyshev smoothing decision and coefficients of an aggregation level (ncol set).
void cheb_setup(HostLevel &L, const lamg_options &o);
int dense_pinv(const HostMat &A, std::vector<double> &pinv);
// In-place inverse of the dense symmetric positive definite n x n row-major M on the GPU
// (dense_kernels.cu, Gauss-Jordan without pivoting); LAMG_ERR_DISCONNECTED when a pivot is not
// positive.
int gpu_dense_inverse(int64_t n, std::vector<double> &M);
double cycle_index(int64_t El, int64_t El1, int64_t E0);

// GPU setup kernels (setup_kernels.cu): K test vectors by colour-ordered GS on A x = 0 and
// the affinity / veto pass. All pointers are host pointers; the functions manage device
// copies themselves. X is n x K row-major.
int gpu_testvectors(const HostMat &A, const std::vector<int32_t> &colour, int level,
                    uint64_t seed, int K, int nu, double *X, int order);
int gpu_affinity(const HostMat &A, const double *X, int K, double tau, double *aff,
                 uint8_t *strong);
// ... and the guard of Eq. 4 per entry (adm[e]: strong and energy ratio <= Q), from the
// moments of Appendix B computed on the GPU.
// Galerkin P^T A P of an aggregation level on the GPU (setup_kernels.cu): ptr/rows/pw is P^T by
// coarse row (galerkin_pt); every coarse entry is the same ordered sum of explicitly rounded
// products as the host's, so Ac equals the host result bit for bit. Rows with more than
// GAL_CAP distinct coarse columns come from host_rows(rows, cols, vals, diags), which fills, for
// each listed coarse row, its nonzero off-diagonal entries in ascending column order and its
// diagonal.
constexpr int GAL_CAP = 128;
using GalerkinHostRows = std::function<void(const std::vector<int64_t> &, std::vector<std::vector<int32_t>> &,
                                            std::vector<std::vector<double>> &, std::vector<double> &)>;
int gpu_galerkin(const HostLevel &L, const std::vector<int64_t> &ptr, const std::vector<int32_t> &rows,
                 const std::vector<double> &pw, HostMat &Ac, const GalerkinHostRows &host_rows);
// Exact Schur complement onto C of an elimination level on the GPU (setup_kernels.cu): row i is
// node cnode[i]; the same ordered, explicitly rounded sums as the host's row, so Ac equals the
// host result bit for bit. Rows with more than GAL_CAP distinct coarse columns come from
// host_rows (as for gpu_galerkin, rows given by coarse index).
int gpu_schur(const HostMat &A, const std::vector<uint8_t> &inF, const std::vector<int32_t> &cidx,
              const std::vector<int32_t> &cnode, HostMat &Ac, const GalerkinHostRows &host_rows);
// The per-entry input checks of validate_graph on the GPU (setup_kernels.cu), for a graph whose
// row pointers start at 0 and never decrease: *valid = every entry passes.
int gpu_validate_entries(const lamg_graph *g, bool *valid);
int gpu_tv_and_affinity(const HostMat &A, const std::vector<int32_t> &colour, int level,
                        uint64_t seed, int K, int nu, double tau, int veto, double *X,
                        double *aff, uint8_t *strong, double Q, double eps, uint8_t *adm, int order,
                        int32_t *choice = nullptr, int *rounds = nullptr);
// With choice != nullptr gpu_tv_and_affinity also runs the aggregation pass of Section 2 on the GPU
// (k_agg_round): choice[u] = the node u joined, or -1 if u is a seed; *rounds = parallel rounds.

int cuda_status(cudaError_t e);

}  // namespace lamg
