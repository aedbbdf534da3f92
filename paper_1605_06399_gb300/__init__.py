"""GB300-native per-pixel stencil operators (ImageCL's method, arXiv 1605.06399)."""
