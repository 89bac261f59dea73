// Expensive-potential kernels with the bf16 hi/lo tensor-core readout
// (k_ace_tc.cuh).
#include "k_ace_tc.cuh"

namespace mixd {

cudaError_t ace_gaunt_upload_tc2(const void* ent_f, int n_ent, const int* rows, int n_rows) {
    return gaunt_upload_module(ent_f, n_ent, rows, n_rows);
}

cudaError_t ace_tc_configure_2(int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid, int* nbuf) {
    return ace_tc_cfg<2>(L, n, cap, tile_max, qb, smem, grid, nbuf);
}

void launch_ace_tc_2(const Dev& d, const AceTab<float>& tab, int L, size_t smem, int grid, int nbuf, cudaStream_t s) {
    ace_tc_launch<2>(d, tab, L, smem, grid, nbuf, s);
}

}  // namespace mixd
