// Ablation-variant kernels with value polynomials of degree 2 (all key sets).
#include "variants.cuh"

namespace efunc {
namespace variant {

EFUNC_VARIANT_DEGREE(2)

}  // namespace variant
}  // namespace efunc
