// Checkpoint files of the IMEX-TR outer loop (host code only; no CUDA).
//
// A checkpoint taken after outer iteration j - 1 holds everything the loop carries into
// iteration j: the iterate v (N doubles) and the scalars of Algorithm 1 (r, nu, mu, the
// previous ratio and whether it exists), the pending random start of the next subproblem
// and the random-stream counter, plus the counters reported in lb_tr_info.  Resuming from
// it repeats the remaining iterations exactly, since every reduction of the library is
// summed in a fixed order.
//
// Files: <path>.npy (the iterate, NumPy format 1.0, little-endian float64, C order
// [z][y][x] or [y][x]) and <path>.json (the scalars; doubles with 17 significant digits).
// Both are written to temporaries and renamed, the JSON last, so a reader never sees a
// JSON file whose field file is missing or older.
#pragma once
#include <string>
#include <vector>

namespace lbtr {

struct TrCheckpoint {
    int dim = 0;
    int n = 0;                  // points per axis
    int j = 0;                  // next outer iteration
    double r = 0.0, nu = 0.0, mu = 0.0, rho_prev = 0.0;
    int have_rho = 0;
    int random_next = 0;
    unsigned rstream = 0;
    int accepted = 0, contracted = 0, shrunk = 0, randomized = 0;
    long long inner = 0;
    double g1_min = 0.0;        // NaN if never measured
    int sub_stalled = 0, sub_capped = 0;
    double sub_worst_rel_res = 0.0;
    // the problem and the solver settings the state belongs to: a resume with other values
    // would carry r, nu, mu and the previous ratio into a different problem
    double box[3] = {0.0, 0.0, 0.0};
    double xi = 0.0, tau = 0.0, gamma = 0.0, eta = 0.0;
    int precision = 0;          // lb_precision of the context
};

// true if `c` (read from a file) was written for the problem and settings of `want`
// (grid, box lengths, xi, tau, gamma, precision and the subproblem step eta, compared
// exactly: they are written with 17 digits); false with a message naming the first mismatch
bool checkpoint_matches(const TrCheckpoint& c, const TrCheckpoint& want, std::string& err);

// false with a message on any I/O error
bool write_checkpoint(const std::string& path, const TrCheckpoint& c, const double* field, long long count,
                      std::string& err);
// false with a message on any I/O or format error (including a field of the wrong size)
bool read_checkpoint(const std::string& path, TrCheckpoint& c, std::vector<double>& field, std::string& err);

}  // namespace lbtr
