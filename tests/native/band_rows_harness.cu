// Host-only harness for the row and column limits of the partial-Cholesky launches
// (BandRows, band_limit, profile_rows in common.cuh): reads one matrix description and a list
// of queries from stdin and prints, per query, the column limit and the rows a launch visits.
//   input:  m e band id0 nq / nq values of ifirst (non-decreasing) / nquery / row0 ke (x nquery)
//   output: per query "lim nv r_0 ... r_{nv-1}"
#include <cstdio>
#include <vector>

#include "common.cuh"

int main() {
  int m, e, band, id0, nq;
  if (std::scanf("%d %d %d %d %d", &m, &e, &band, &id0, &nq) != 5) return 1;
  std::vector<int> q(nq);
  for (int i = 0; i < nq; ++i)
    if (std::scanf("%d", &q[i]) != 1) return 1;
  bd::MatDesc d{0, m, m, e, 0};
  d.band = band;
  d.id0 = id0;
  d.ifirst = nq > 0 ? q.data() : nullptr;
  int nquery;
  if (std::scanf("%d", &nquery) != 1) return 1;
  for (int t = 0; t < nquery; ++t) {
    int row0, ke;
    if (std::scanf("%d %d", &row0, &ke) != 2) return 1;
    const bd::BandRows br = bd::band_rows(d, row0, ke);
    std::printf("%d %d", bd::band_limit(d, ke), br.nv);
    for (int v = 0; v < br.nv; ++v) std::printf(" %d", br.row(v));
    std::printf("\n");
  }
  return 0;
}
