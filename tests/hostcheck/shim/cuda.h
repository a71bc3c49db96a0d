// Test double of the one driver-API type the batched engine's descriptors
// name (CUtensorMap), so that batched.cpp compiles for the host test library.
// TEST INFRASTRUCTURE ONLY: never part of the product library.
#pragma once
#include "cuda_runtime.h"

struct alignas(64) CUtensorMap {
    unsigned long long opaque[16];
};
