"""GB300-native DG-MHD hot path (modal DG, ideal MHD, Powell/LDF or GLM)."""
