// Limits shared by the training translation unit and its callers.
#pragma once
#include "../../include/eventtracer.h"

constexpr int kMaxSeg = 32;   // longest BPTT segment (membrane checkpoint interval)
