// Host dump of the library's table blob (csrc/nir_basis.cpp, layout of
// csrc/nir_layout.h) for the CPU test tests/test_tables_cpu.py.  Not part of
// the library.  argv: shape P; stdout: the layout offsets
// (Ba Bb Bc D1 D2 D3 wq Bs total), then the blob.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "nir_basis.h"
#include "nir_layout.h"

int main(int argc, char **argv)
{
    if (argc != 3) return 2;
    const int shape = std::atoi(argv[1]), P = std::atoi(argv[2]), N = P + 1, Q = P + 2;
    const nirk::TabLayout L = nirk::layout(shape, N, Q);
    std::vector<double> blob(L.total);
    if (nirb_table_size(shape, P, Q) != L.total || !nirb_build_tables(shape, P, Q, blob.data(), 0)) return 3;
    std::printf("%d %d %d %d %d %d %d %d %d\n", L.Ba, L.Bb, L.Bc, L.D1, L.D2, L.D3, L.wq, L.Bs, L.total);
    for (double v : blob) std::printf("%.17g\n", v);
    return 0;
}
