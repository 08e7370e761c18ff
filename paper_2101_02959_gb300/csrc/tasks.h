// Plain-data task descriptors shared by the host orchestration and the kernels.
#pragma once

namespace bd {

// Block copy: dst[i][k] = sign * src(...), i < rows, k < cols.
//   mode 0: src[r0 + i][c0 + k]
//   mode 1: src[r0 + k][c0 + i]              (transpose)
//   mode 2: src[r0 + max(i,k)][c0 + min(i,k)] (symmetric matrix from its lower triangle)
//   mode 3: as mode 2, reading only lower entries (coalesced) and writing both halves
struct CopyTask {
  long long src_off, dst_off;
  int src_ld, dst_ld, r0, c0, rows, cols, mode, pad;
  double sign;
};

// C = A B for n x n blocks (A, B with leading dimension n; C with ldc).
struct GemmTask {
  long long a_off, b_off, c_off;
  int n, ldc;
};

// One dual class (deluxe scaling, Section 4.2).
struct ClassTask {
  long long sinv_off;  // (sum_m S_C^(m))^-1, n x n
  int n;               // dual dofs of the class
  int dual_start;      // first global transformed dual dof
  int pair_beg, pair_end;
};

// One (class, subdomain) pair: the principal minor S_C^(j) and its place in
// the subdomain's local dual vector (concatenated over subdomains).
struct PairTask {
  long long blk_off;
  int ldual_off;
  int sub;
};

// One FETI-DP multiplier block lambda_{ab} on a class (a < b in N_C).
struct LamTask {
  int lam_off, n;
  int pa, pb;          // PairTask indices of subdomains a and b
  long long sinv_off;
};

// One (subdomain, class) block of a local dual vector and the multipliers touching it.
struct WTask {
  long long sinv_off;
  int ldual_off, n;
  int ent_beg, ent_end;
};
struct WEnt {
  long long partner_blk_off;  // S_C^(partner)
  int lam_off;
  int sign;                   // +1 if this subdomain is the first of the pair
};

}  // namespace bd
