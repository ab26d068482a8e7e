// FP32 mesh / FFT / particle path (FP64 reductions): explicit instantiation.
#include "rom.cuh"

template struct pm::Engine<float>;
template struct pm::rom::Rom<float>;
