// Internal declarations shared by the host lattice code and the CUDA solver.
#pragma once

#include <cstdint>
#include <string>

#include "../../include/fftHomog.h"

namespace fh {

// Thread-local error text behind fh_last_error().
void set_error(const std::string& msg);

// Exact description of one pattern P(M) (Sec. 2.1 of the paper).
//
// Smith normal form U M V = diag(snf), U, V unimodular.  Non-trivial axes
// (snf > 1) become the storage axes k = 0..nd-1, in increasing length, the
// last one contiguous; axis_of[k] is the SNF index of storage axis k.
struct Pattern {
  int d = 0;
  int64_t M[3][3] = {};
  int64_t adj[3][3] = {};   // adj(M):   M^-1   = adj  / det
  int64_t adjT[3][3] = {};  // adj(M^T): M^-T   = adjT / det
  int64_t D = 0;            // m = |det M|
  int sign = 1;             // sign of det M
  int64_t U[3][3] = {}, Uinv[3][3] = {}, V[3][3] = {}, Vinv[3][3] = {};
  int64_t snf[3] = {1, 1, 1};
  int nd = 0;
  int dims[3] = {1, 1, 1};
  int axis_of[3] = {0, 0, 0};
  // Storage axis k, index n_k, contributes n_k * Pmap[k][.] to j = U^-1 n
  // and l_k * Fmap[k][.] to h = V^-T l (before reduction).
  int64_t Pmap[3][3] = {};
  int64_t Fmap[3][3] = {};

  int64_t half_len() const;  // dims_last / 2 + 1
  int64_t n_half() const;    // number of stored half-spectrum frequencies
  // exact maps (host)
  void point_numerator(int64_t storage_index, int64_t* a) const;
  void half_freq(int64_t half_index, int64_t* h) const;
};

fh_status build_pattern(int d, const int64_t* M, Pattern* out);

// FFT length plan: L = r_0 r_1 ... r_{np-1}, radices in {2,3,4,5,7,8,11,13}.
struct FftPlan {
  int L = 1;
  int np = 0;
  int r[24] = {};
};
bool make_plan(int L, FftPlan* plan);

}  // namespace fh

struct fh_pattern {
  fh::Pattern p;
};
