// Ablation-variant kernels with value polynomials of degree 0 (all key sets).
#include "variants.cuh"

namespace efunc {
namespace variant {

EFUNC_VARIANT_DEGREE(0)

}  // namespace variant
}  // namespace efunc
