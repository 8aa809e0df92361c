// Test driver: writes the library's canonical node positions and Dirichlet
// flags of one shell level as raw binary, for comparison with the oracle.
// usage: mesh_dump r1 r2 tang layers N out.bin
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1608_06473_gb300/csrc/mesh.h"

int main(int argc, char** argv) {
  if (argc != 7) return 2;
  const double r1 = atof(argv[1]), r2 = atof(argv[2]);
  const int tang = atoi(argv[3]), layers = atoi(argv[4]), N = atoi(argv[5]);
  hhg::MacroMesh m = hhg::build_shell(r1, r2, tang, layers);
  hhg::LevelLayout lay = hhg::make_layout(m, N);
  std::vector<double> xyz(3 * lay.n_total);
  hhg::level_coords(m, lay, xyz.data());
  std::vector<unsigned char> dir(lay.n_total);
  for (int64_t i = 0; i < lay.n_total; ++i) dir[i] = hhg::node_dirichlet(m, lay, i);
  FILE* f = fopen(argv[6], "wb");
  const int64_t hdr[6] = {lay.n_total, lay.nV, lay.nE, lay.nF, lay.nC, lay.off_C};
  fwrite(hdr, sizeof(hdr), 1, f);
  fwrite(xyz.data(), sizeof(double), xyz.size(), f);
  fwrite(dir.data(), 1, dir.size(), f);
  // cell-local canonical maps of the first cells (full tets)
  for (int c = 0; c < (int)m.cells.size(); ++c)
    for (int k = 0; k <= N; ++k)
      for (int j = 0; j <= N - k; ++j)
        for (int i = 0; i <= N - j - k; ++i) {
          const int64_t idx = hhg::cell_node_index(m, lay, c, i, j, k);
          fwrite(&idx, sizeof(idx), 1, f);
        }
  fclose(f);
  return 0;
}
