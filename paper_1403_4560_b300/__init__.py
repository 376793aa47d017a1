"""sgmc: B300-native Monte Carlo engine for the 3D Edwards-Anderson spin glass
in a field (arXiv:1403.4560). The compute path is libsgmc.so (CUDA, sm_103a);
`sgmc` is its ctypes binding and `inputs` holds the seeded synthetic inputs."""
