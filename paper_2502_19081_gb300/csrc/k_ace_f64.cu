// Expensive-potential kernel instantiations with double arithmetic (the
// templates and their description are in k_ace.cuh).
#include "k_ace.cuh"

namespace mixd {

cudaError_t ace_configure_f64(int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid, int wn) {
    return ace_cfg_t<double>(false, L, n, cap, tile_max, qb, smem, grid, wn);
}

void launch_ace_f64(const Dev& d, const void* tab, int L, size_t smem, int grid, int wn, cudaStream_t s) {
    ace_launch_t<double>(d, *static_cast<const AceTab<double>*>(tab), L, smem, grid, wn, s);
}

cudaError_t ace_batch_configure_f64(int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid) {
    return ace_cfg_t<double>(true, L, n, cap, tile_max, qb, smem, grid);
}

void launch_ace_batch_f64(const Dev* devs, const void* tabs, const int2* list, const int* count, int n, int L,
                          size_t smem, int grid, cudaStream_t s) {
    AceBatch<double> b{devs, static_cast<const AceTab<double>*>(tabs), list, count};
    ace_batch_launch_t<double>(b, n, L, smem, grid, s);
}

cudaError_t ace_configure(int precision, int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid,
                          int wn) {
    if (cap > MAX_CAP || n > 16 || qb < 1 || (wn != ACE_GROUP && wn != ACE_MAX_WARPS)) return cudaErrorInvalidValue;
    return precision == MIX_FP64 ? ace_configure_f64(L, n, cap, tile_max, qb, smem, grid, wn)
                                 : ace_configure_f32(L, n, cap, tile_max, qb, smem, grid, wn);
}

cudaError_t ace_gaunt_upload(const void* ent_f, int n_ent, const int* rows, int n_rows) {
    cudaError_t e = ace_gaunt_upload_f32(ent_f, n_ent, rows, n_rows);
    if (e == cudaSuccess) e = ace_gaunt_upload_tc1(ent_f, n_ent, rows, n_rows);
    if (e == cudaSuccess) e = ace_gaunt_upload_tc2(ent_f, n_ent, rows, n_rows);
    return e;
}

void launch_ace(const Dev& d, const void* tab, int precision, int L, size_t smem, int grid, int wn, cudaStream_t s) {
    if (precision == MIX_FP64) launch_ace_f64(d, tab, L, smem, grid, wn, s);
    else launch_ace_f32(d, tab, L, smem, grid, wn, s);
}

}  // namespace mixd

namespace mixd {

cudaError_t ace_batch_configure(int precision, int L, int n, int cap, int tile_max, int qb, size_t* smem, int* grid) {
    if (cap > MAX_CAP || n > 16 || qb < 1) return cudaErrorInvalidValue;
    return precision == MIX_FP64 ? ace_batch_configure_f64(L, n, cap, tile_max, qb, smem, grid)
                                 : ace_batch_configure_f32(L, n, cap, tile_max, qb, smem, grid);
}

void launch_ace_batch(int precision, const Dev* devs, const void* tabs, const int2* list, const int* count, int n,
                      int L, size_t smem, int grid, cudaStream_t s) {
    if (precision == MIX_FP64) launch_ace_batch_f64(devs, tabs, list, count, n, L, smem, grid, s);
    else launch_ace_batch_f32(devs, tabs, list, count, n, L, smem, grid, s);
}

}  // namespace mixd
