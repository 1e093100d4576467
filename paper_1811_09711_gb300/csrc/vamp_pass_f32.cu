// FP32-eval pass kernels for any shape (d <= 16, n <= 256).
#include "vamp_pass.cuh"

namespace vamp {
void add_pass_variants_f32_generic(std::vector<PassVariant>& v)
{
    v.push_back(make_variant<float, 2, 0, 0>());
}
}  // namespace vamp
