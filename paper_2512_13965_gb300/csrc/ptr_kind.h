// Classification of a caller's array by where it lives, from the fields of
// cudaPointerAttributes. Plain C++ with no CUDA headers, so a host-only unit
// test checks every case without a GPU.
#pragma once

namespace gmc {

enum PtrKind {
  kPtrDevice = 0,       // device memory of the context's GPU, or managed memory
  kPtrOtherDevice = 1,  // device memory of another GPU: rejected (a kernel here would
                        // read it over the peer link or fault when peer access is off)
  kPtrMappedHost = 2,   // page-locked host memory with a device address: used in place
  kPtrHost = 3,         // any other host memory: staged through context buffers
};

// mem_type: the cudaMemoryType value (0 unregistered, 1 host, 2 device,
// 3 managed); ptr_device: the attribute's device; ctx_device: the context's
// device; has_device_address: whether the attribute's devicePointer is set.
inline PtrKind classify_pointer(int mem_type, int ptr_device, int ctx_device,
                                bool has_device_address) {
  switch (mem_type) {
    case 2: return ptr_device == ctx_device ? kPtrDevice : kPtrOtherDevice;
    case 3: return kPtrDevice;
    case 1: return has_device_address ? kPtrMappedHost : kPtrHost;
    default: return kPtrHost;
  }
}

}  // namespace gmc
