// Plane-kernel instantiations for double (one translation unit per precision).
#include "plane_ops.cuh"

namespace tddft {

template <>
PlaneOps<double> plane_ops_for<double>(int n) {
  switch (n) {
    case 8:
      return PlaneLaunch<double, 8>::ops();
    case 12:
      return PlaneLaunch<double, 12>::ops();
    case 16:
      return PlaneLaunch<double, 16>::ops();
    case 24:
      return PlaneLaunch<double, 24>::ops();
    case 32:
      return PlaneLaunch<double, 32>::ops();
    case 36:
      return PlaneLaunch<double, 36>::ops();
    case 48:
      return PlaneLaunch<double, 48>::ops();
    case 64:
      return PlaneLaunch<double, 64>::ops();
    case 72:
      return PlaneLaunch<double, 72>::ops();
    case 80:
      return PlaneLaunch<double, 80>::ops();
    case 96:
      return PlaneLaunch<double, 96>::ops();
    case 108:
      return PlaneLaunch<double, 108>::ops();
    default:
      return PlaneOps<double>{};
  }
}

}  // namespace tddft
