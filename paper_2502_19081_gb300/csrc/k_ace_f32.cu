// Expensive-potential kernel instantiations with float arithmetic (the
// templates and their description are in k_ace.cuh).
#include "k_ace.cuh"

namespace mixd {

cudaError_t ace_gaunt_upload_f32(const void* ent_f, int n_ent, const int* rows, int n_rows) {
    return gaunt_upload_module(ent_f, n_ent, rows, n_rows);
}

cudaError_t ace_configure_f32(int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid, int wn) {
    return ace_cfg_t<float>(false, L, n, cap, tile_max, qb, smem, grid, wn);
}

void launch_ace_f32(const Dev& d, const void* tab, int L, size_t smem, int grid, int wn, cudaStream_t s) {
    ace_launch_t<float>(d, *static_cast<const AceTab<float>*>(tab), L, smem, grid, wn, s);
}

cudaError_t ace_batch_configure_f32(int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid) {
    return ace_cfg_t<float>(true, L, n, cap, tile_max, qb, smem, grid);
}

void launch_ace_batch_f32(const Dev* devs, const void* tabs, const int2* list, const int* count, int n, int L,
                          size_t smem, int grid, cudaStream_t s) {
    AceBatch<float> b{devs, static_cast<const AceTab<float>*>(tabs), list, count};
    ace_batch_launch_t<float>(b, n, L, smem, grid, s);
}

}  // namespace mixd
