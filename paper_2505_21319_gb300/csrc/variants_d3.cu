// Ablation-variant kernels with value polynomials of degree 3 (all key sets).
#include "variants.cuh"

namespace efunc {
namespace variant {

EFUNC_VARIANT_DEGREE(3)

}  // namespace variant
}  // namespace efunc
