// Reverse-mode launchers, double.
#include "adj_impl.cuh"

MPA_ADJ_INSTANTIATE(double)
