"""GB300-native gamblet multiresolution solver (Owhadi, Sec. 4-5).

``native`` is the thin ctypes binding of libgamblet.so (include/gamblet.h);
``solver`` wraps it in a handle class and a torch.autograd.Function.
Importing either loads the CUDA library; it must have been built first
(``python -m paper_1503_03467_gb300.build``).
"""
