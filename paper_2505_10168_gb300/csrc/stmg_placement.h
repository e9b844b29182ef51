// stmg_placement.h -- the pointer-placement rule of the library's device-array checks
// (stmg_sensitivity_noalloc, and every call that reads a caller's array in place), kept free
// of CUDA calls so that host-only tests can compile and check it.
//
// type is the cudaMemoryType that cudaPointerGetAttributes reports for a pointer
// (0 unregistered host, 1 registered host, 2 device, 3 managed), device its device
// ordinal, current the caller's current device.  Managed memory is reachable from any
// device; device memory only from its own device (the library enables no peer access).
#pragma once

namespace stmg {

enum { kPlaceUsable = 0, kPlaceOtherDevice = 1, kPlaceNotDevice = 2 };

inline int noalloc_placement(int type, int device, int current) {
  if (type == 3) return kPlaceUsable;
  if (type != 2) return kPlaceNotDevice;
  return device == current ? kPlaceUsable : kPlaceOtherDevice;
}

}  // namespace stmg
