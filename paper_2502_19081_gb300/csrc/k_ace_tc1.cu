// Expensive-potential kernels with the bf16 tensor-core readout (k_ace_tc.cuh),
// and the dispatch of both readout variants.
#include "k_ace_tc.cuh"

namespace mixd {

cudaError_t ace_gaunt_upload_tc1(const void* ent_f, int n_ent, const int* rows, int n_rows) {
    return gaunt_upload_module(ent_f, n_ent, rows, n_rows);
}

cudaError_t ace_tc_configure_2(int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid, int* nbuf);
void launch_ace_tc_2(const Dev& d, const AceTab<float>& tab, int L, size_t smem, int grid, int nbuf, cudaStream_t s);

cudaError_t ace_tc_configure(int tcm, int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid,
                             int* nbuf) {
    if (cap > MAX_CAP || n > 16 || qb < 1 || L < 0 || L > 6) return cudaErrorInvalidValue;
    if (tcm == 1) return ace_tc_cfg<1>(L, n, cap, tile_max, qb, smem, grid, nbuf);
    if (tcm == 2) return ace_tc_configure_2(L, n, cap, tile_max, qb, smem, grid, nbuf);
    return cudaErrorInvalidValue;
}

void launch_ace_tc(const Dev& d, const void* tab, int tcm, int L, size_t smem, int grid, int nbuf, cudaStream_t s) {
    const AceTab<float>& t = *static_cast<const AceTab<float>*>(tab);
    if (tcm == 1) ace_tc_launch<1>(d, t, L, smem, grid, nbuf, s);
    else launch_ace_tc_2(d, t, L, smem, grid, nbuf, s);
}

}  // namespace mixd
