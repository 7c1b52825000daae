// CPU check of the host graph builders (csrc/sg_graph_build.h): reads a CSR
// (n, m, row_ptr int64[n+1], col int32[m]) from argv[1], builds the
// canonical CSR and the CSC with argv[3] host threads, writes
// rp_out, col_out, crp, cin (int32 arrays, with their lengths) to argv[2].
#include <stdio.h>
#include <stdlib.h>

#include "sg_graph_build.h"

int main(int argc, char **argv)
{
    if (argc != 4) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 3;
    int64_t nm[2];
    if (fread(nm, 8, 2, f) != 2) return 4;
    const int64_t n = nm[0], m = nm[1];
    std::vector<int64_t> rp((size_t)n + 1);
    std::vector<int32_t> col((size_t)(m > 0 ? m : 1));
    if (fread(rp.data(), 8, (size_t)n + 1, f) != (size_t)n + 1) return 5;
    if (m && fread(col.data(), 4, (size_t)m, f) != (size_t)m) return 6;
    fclose(f);
    sgh::thread_cap() = atoi(argv[3]);
    const int64_t bad = sgh::parallel_first(m, [&](int64_t e) { return col[(size_t)e] < 0 || col[(size_t)e] >= n; });
    if (bad < m) return 7;
    sgh::hvec<int32_t> rpc, colc, crp;
    sgh::hvec<sgh::Arc2> cin;
    sgh::canonicalise(n, rp.data(), col.data(), rpc, colc);
    sgh::build_csc(n, rpc, colc, crp, cin);
    const int64_t mc = rpc[(size_t)n];
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 8;
    fwrite(&mc, 8, 1, o);
    fwrite(rpc.data(), 4, (size_t)n + 1, o);
    fwrite(colc.data(), 4, (size_t)mc, o);
    fwrite(crp.data(), 4, (size_t)n + 1, o);
    fwrite(cin.data(), 8, (size_t)mc, o);
    fclose(o);
    return 0;
}
