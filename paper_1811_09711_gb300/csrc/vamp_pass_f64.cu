// FP64 pass kernels for any shape (d <= 16, n <= 256).
#include "vamp_pass.cuh"

namespace vamp {
void add_pass_variants_f64(std::vector<PassVariant>& v)
{
    v.push_back(make_variant<double, 1, 0, 0>());
}
}  // namespace vamp
