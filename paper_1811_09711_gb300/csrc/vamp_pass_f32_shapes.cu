// FP32-eval pass kernels specialised for fixed shapes (d, n): the collider
// workload (14, 100) and the small reference problems (8, 50), (4, 20).
// Every block offset is a compile-time constant in these kernels.
#include "vamp_pass.cuh"

namespace vamp {
void add_pass_variants_f32_shapes(std::vector<PassVariant>& v)
{
    v.push_back(make_variant<float, 2, 14, 100>());
    v.push_back(make_variant<float, 4, 14, 100>());
    v.push_back(make_variant<float, 1, 14, 100, 3>());
    v.push_back(make_variant<float, 2, 14, 100, 3>());
    v.push_back(make_variant<float, 1, 14, 100, 4>());
    v.push_back(make_variant<float, 4, 8, 50>());
    v.push_back(make_variant<float, 4, 4, 20>());
}
}  // namespace vamp
