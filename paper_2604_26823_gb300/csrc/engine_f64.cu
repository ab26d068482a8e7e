// All-FP64 path: explicit instantiation.
#include "rom.cuh"

template struct pm::Engine<double>;
template struct pm::rom::Rom<double>;
