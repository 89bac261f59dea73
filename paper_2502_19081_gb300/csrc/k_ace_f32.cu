// Expensive-potential kernel instantiations with float arithmetic (the
// templates and their description are in k_ace.cuh).
#include "k_ace.cuh"

namespace mixd {

cudaError_t ace_configure_f32(int L, int n, int cap, size_t* smem, int* grid) {
    return ace_cfg_t<float>(L, n, cap, smem, grid);
}

void launch_ace_f32(const Dev& d, const void* tab, int L, size_t smem, int grid, cudaStream_t s) {
    ace_launch_t<float>(d, *static_cast<const AceTab<float>*>(tab), L, smem, grid, s);
}

}  // namespace mixd
