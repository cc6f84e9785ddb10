"""B300-native simulator of N coupled spin-torque oscillators (arXiv 2312.01121)."""
